"""The paper's characterisation experiments, re-run on B300 with the library's kernels.

    python -m paper_2501_16909_b300.experiments [names ...] [--repeats R] [--out results.json]

Each experiment is the B300 counterpart of one measurement of the paper, built from
the library's stressors and victims through the C ABI (no vLLM, cuBLAS or MPS):

  pitfall1  Sec. 3, Pitfall 1: two compute kernels of one 128-thread block per SM
            (the paper's 6.25 % achieved occupancy): (a) one of them squeezed onto
            6.25 % of the SMs with the same total work, (b) both colocated on all SMs.
  pitfall2  Sec. 3, Pitfall 2: a compute kernel (one 512-thread block per SM, ILP 8:
            four warps per sub-partition, enough to issue an FFMA every cycle) beside a
            copy kernel over 4 GiB (one 1024-thread block per SM) with similar solo
            time: each one's slowdown and the compute kernel's issue rate.  The paper
            used 1024 threads for both; here that would need 73 728 registers per SM
            (40 + 32 per thread), so the pair could not share an SM at all.
  ipc       Sec. 4.4.2, Table 2: the compute kernel at S1..S4 (ILP 1, 2, 4, 8; one
            128-thread block per SM) beside memory-bound victims: its solo issue rate
            and each victim's slowdown.
  fp64      Sec. 4.4.3, Table 3: two fp64 compute kernels at S1..S4 (ILP 1..4, one
            128-thread block per SM): solo fp64-pipe utilisation and issue rate, and
            the speedup of running them together over running them back to back.
  l2        Sec. 4.3, Fig. 3: two copy kernels on disjoint SM halves over growing
            per-instance data: one kernel's slowdown against alone, and its solo rate.
  l2_green  the same with the halves as two green-context partitions (the paper's
            mechanism) instead of explicit SM masks.
  smem      Sec. 4.4.1, Fig. 4: BF16 GEMM victims (1024^3, 2048^3, 4096^3) beside the
            n-strided shared-memory stressor, n = 1, 2, 4, ..., 32: slowdown per n.
  bandwidth Sec. 4.3, Table 1: victims in one green-context partition (half the SMs)
            beside a copy kernel in the other, 512-thread blocks on half its SMs, then 1,
            2 and 3 per SM: victim slowdown and the copy's HBM bandwidth.
  variants  Sec. 5.3, colocation-friendly kernel variants: the BF16 GEMM with 3 TMA
            stages (145 KiB of shared memory) and with 4 (193 KiB), alone and arriving
            at each full-SM stressor: solo throughput against latency beside it.  (The
            CTA-pair variant is left out: its paired TMEM allocation can wait for the
            tensor stressor to end.)
  decode    Tables 1 and 2 in the paper's terms: one synthetic decoder layer's decode
            kernels (batch 64, KV length 4096, hidden 4096) as the victim set, (a) beside
            the compute kernel at S1..S4 on the same SMs, (b) in one green-context
            partition beside the copy kernel in the other; per-kernel slowdowns (Fig. 5)
            and the layer's step latency (the sum of its kernels' per-launch times).
  hol       Sec. 4.2, block-scheduler interference: a 10 ms sleep kernel (one 128-thread
            block per SM) released together with victims of small and large per-block
            footprints: victim latency from the release, alone and beside it, and
            whether its first block had to wait for the sleep kernel to leave.

Issue rates are warp instructions of the kernel's arithmetic (FFMA or DMUL) per cycle
per SM at the maximum SM clock; the loop's few other instructions are not counted.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch  # noqa: E402

import ifr_inputs as I  # noqa: E402

from . import _abi as A  # noqa: E402
from . import peaks as P  # noqa: E402
from . import stressor_cfg, victim_cfg  # noqa: E402

GiB = 1 << 30
MiB = 1 << 20


# ----------------------------------------------------------------------------- helpers
def mask_bits(sm_ids):
    """ifr_stressor_cfg.sm_mask words for a set of SM ids (mask_mode 2)."""
    words = [0] * (A.IFR_MAX_SMS // 32)
    for s in sm_ids:
        words[s >> 5] |= 1 << (s & 31)
    return words


def with_mask(cfg, sm_ids):
    ids = sorted(set(sm_ids))
    cfg.mask_mode = 2
    cfg.sm_count = len(ids)
    for i, w in enumerate(mask_bits(ids)):
        cfg.sm_mask[i] = w
    return cfg


def issue_rate(rate_ops, S, clk_hz):
    """Warp instructions per cycle per SM for `rate_ops` thread-level operations per s."""
    return rate_ops / 32.0 / (S * clk_hz)


def pair_stats(runs):
    """Medians over repeated ifr_stressor_pair results."""
    med = lambda k: statistics.median(r[k] for r in runs)
    return {
        "solo_a_us": med("solo_a_ns") / 1e3, "solo_b_us": med("solo_b_ns") / 1e3,
        "co_a_us": med("co_a_ns") / 1e3, "co_b_us": med("co_b_ns") / 1e3,
        "slowdown_a": statistics.median(r["co_a_ns"] / r["solo_a_ns"] for r in runs),
        "slowdown_b": statistics.median(r["co_b_ns"] / r["solo_b_ns"] for r in runs),
        "speedup_seq_over_col": statistics.median(r["seq_ns"] / r["col_ns"] for r in runs),
        "all_overlapped": all(r["overlapped"] for r in runs),
        "all_ok": all(r["status"] == A.IFR_OK for r in runs),
    }


def run_pair(ctx, a, b, repeats):
    return pair_stats([ctx.stressor_pair(a, b) for _ in range(repeats)])


def fixed_span_us(ctx, cfg):
    res, _ = ctx.run_stressor(cfg, 30000)
    return (res["t_end_ns"] - res["t_start_ns"]) / 1e3, res


def slowdowns_from_cells(cells, n_victims, n_levels):
    """Per victim: [slowdown at level 0..n_levels] = median measured time / median solo."""
    per = lambda t: (t.t_end_ns - t.t_start_ns) / max(1, t.repeats)
    out = []
    for v in range(n_victims):
        solo = [per(c.timing) for c in cells if c.victim == v and c.stressor < 0 and c.valid]
        t0 = statistics.median(solo)
        row = []
        for lv in range(n_levels + 1):
            xs = [per(c.timing) for c in cells if c.victim == v and c.stressor == 0 and c.level == lv and c.valid]
            row.append(round(statistics.median(xs) / t0, 3) if xs else None)
        out.append({"solo_us": round(t0 / 1e3, 2), "slowdown": row})
    return out


# ----------------------------------------------------------------------------- experiments
def exp_pitfall1(ctx, repeats):
    S = ctx.info["num_sms"]
    rounds = 64
    base = dict(block=128, blocks_per_sm=1, ilp=4, max_rounds=rounds)
    full = stressor_cfg(A.IFR_S_FMA, sm_count=S, seed=1, **base)
    t_full = statistics.median(fixed_span_us(ctx, full)[0] for _ in range(repeats))
    # (a) the same S blocks' work on 6.25 % of the SMs, 16 blocks per SM (2048 threads)
    n = max(1, round(0.0625 * S))
    bps = min(16, math.ceil(S / n))
    sq_rounds = max(1, round(rounds * S / (n * bps)))
    squeezed = stressor_cfg(A.IFR_S_FMA, sm_count=n, seed=1, block=128, blocks_per_sm=bps, ilp=4,
                            max_rounds=sq_rounds)
    t_sq = statistics.median(fixed_span_us(ctx, squeezed)[0] for _ in range(repeats))
    work_ratio = (n * bps * sq_rounds) / (S * rounds)
    # (b) two instances on all SMs
    other = stressor_cfg(A.IFR_S_FMA, sm_count=S, seed=2, **base)
    pr = run_pair(ctx, full, other, repeats)
    return {
        "experiment": "pitfall1", "paper": "Sec. 3 Pitfall 1 (H100: 8.57x squeezed, 1.73x colocated)",
        "kernel": "FMA chains, ILP 4, one 128-thread block per SM (4 of 64 warps: 6.25 % occupancy)",
        "full_sms_us": round(t_full, 1),
        "squeezed": {"sms": n, "blocks_per_sm": bps, "rounds": sq_rounds, "work_ratio": round(work_ratio, 4),
                     "us": round(t_sq, 1), "latency_increase": round(t_sq / t_full / work_ratio, 3)},
        "colocated": pr,
    }


def exp_pitfall2(ctx, repeats, hbm_buf):
    S = ctx.info["num_sms"]
    clk = ctx.info["sm_clock_khz"] * 1e3
    copy = stressor_cfg(A.IFR_S_HBM, sm_count=S, blocks_per_sm=1, block=1024, buf=hbm_buf,
                        working_set_bytes=hbm_buf.numel() * 4, seed=1, max_rounds=512)
    t_copy, _ = fixed_span_us(ctx, copy)
    comp = stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=1, block=512, ilp=8, seed=3, max_rounds=4)
    t_c, _ = fixed_span_us(ctx, comp)
    comp.max_rounds = max(1, round(4 * t_copy / t_c))  # similar solo times, as in the paper
    rate, _ = P.solo_rate(ctx, comp, rounds=comp.max_rounds)
    pr = run_pair(ctx, comp, copy, repeats)
    return {
        "experiment": "pitfall2", "paper": "Sec. 3 Pitfall 2 (H100: copy latency doubles; compute IPC 3.99)",
        "compute": "FMA chains, ILP 8, one 512-thread block per SM, %d rounds" % comp.max_rounds,
        "copy": "stream read of a 4 GiB set, one 1024-thread block per SM, 512 rounds (5 GB)",
        "compute_issue_rate": round(issue_rate(rate / 2, S, clk), 3),
        "slowdown_compute": pr["slowdown_a"], "slowdown_copy": pr["slowdown_b"], "pair": pr,
    }


def _decode_victims():
    t = {}
    R = 8192
    t["vA"] = I.torch_normal_bf16(13, R * R, "cuda").view(R, R)
    t["vx"] = I.torch_normal_bf16(14, R, "cuda")
    t["vy"] = torch.empty(R, device="cuda")
    t["sx"] = I.torch_uniform_pm1(16, 2048 * 4096, "cuda").view(2048, 4096)
    t["sy"] = torch.empty_like(t["sx"])
    t["lx"] = I.torch_uniform_pm1(15, 16384 * 4096, "cuda").view(16384, 4096)
    t["ly"] = torch.empty_like(t["lx"])
    victims = [
        ("gemv 8192x8192", victim_cfg(A.IFR_V_GEMV, t["vA"], t["vx"], t["vy"], m=R, k=R, repeats=16)),
        ("softmax 2048x4096", victim_cfg(A.IFR_V_SOFTMAX, t["sx"], None, t["sy"], m=2048, n=4096, repeats=16)),
        ("layernorm 16384x4096", victim_cfg(A.IFR_V_LAYERNORM, t["lx"], None, t["ly"], m=16384, n=4096, repeats=4)),
    ]
    return victims, t


def exp_ipc(ctx, repeats):
    S = ctx.info["num_sms"]
    clk = ctx.info["sm_clock_khz"] * 1e3
    victims, _t = _decode_victims()
    ilps = [1, 2, 4, 8]
    row = [stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=1, block=128, ilp=i, seed=4, deadline_ns=2 * 10**9)
           for i in ilps]
    ipc = []
    for c in row:
        rate, _ = P.solo_rate(ctx, c, rounds=32)
        ipc.append(round(issue_rate(rate / 2, S, clk), 3))
    cells = ctx.sweep([v for _, v in victims], [row], repeats=repeats, batched=False)
    sl = slowdowns_from_cells(cells, len(victims), len(row))
    return {
        "experiment": "ipc", "paper": "Sec. 4.4.2 Table 2 (RTX3090: compute IPC 1.18 / 2.06 / 2.9 / 3.45 for S1-S4)",
        "scenarios": ["S%d (ILP %d)" % (i + 1, x) for i, x in enumerate(ilps)],
        "compute_issue_rate": ipc,
        "victims": [{"victim": name, **s} for (name, _), s in zip(victims, sl)],
        "note": "slowdown[0] is the zero-SM stressor (harness only); slowdown[i] is scenario S_i",
    }


def exp_fp64(ctx, repeats, fp64_peak):
    S = ctx.info["num_sms"]
    clk = ctx.info["sm_clock_khz"] * 1e3
    rows = []
    for ilp in (1, 2, 4, 8):
        a = stressor_cfg(A.IFR_S_FP64, sm_count=S, blocks_per_sm=1, block=128, ilp=ilp, seed=5, max_rounds=8)
        b = stressor_cfg(A.IFR_S_FP64, sm_count=S, blocks_per_sm=1, block=128, ilp=ilp, seed=6, max_rounds=8)
        rate, _ = P.solo_rate(ctx, a, rounds=8)
        pr = run_pair(ctx, a, b, repeats)
        rows.append({"ilp": ilp, "issue_rate": round(issue_rate(rate, S, clk), 4),
                     "fp64_pipe_util": round(rate / fp64_peak, 4), "dmul_per_s": rate,
                     "speedup_seq_over_col": round(pr["speedup_seq_over_col"], 3), "pair": pr})
    # ncu names one "shared pipe (fp64 + tensor)" on this part: does the fp64 kernel
    # also slow tensor-core work?  The GEMM arriving at a running fp64 kernel (~8 ms).
    G = 4096
    gA = I.torch_normal_bf16(11, G * G, "cuda").view(G, G)
    gB = I.torch_normal_bf16(12, G * G, "cuda").view(G, G)
    gC = torch.empty(G, G, device="cuda")
    gemm = victim_cfg(A.IFR_V_GEMM, gA, gB, gC, m=G, n=G, k=G, repeats=4)
    beside = {}
    for ilp in (1, 4):
        sc = stressor_cfg(A.IFR_S_FP64, sm_count=S, blocks_per_sm=1, block=128, ilp=ilp, seed=5)
        t8 = P.solo_rate(ctx, sc, rounds=8)[1]["elapsed_ms"]
        sc.max_rounds = max(1, round(8 * 8.0 / max(t8, 1e-3)))
        runs = [ctx.colocate(sc, gemm) for _ in range(repeats)]
        beside["ilp%d" % ilp] = {"latency_ratio": round(statistics.median(r["victim_co_ns"] / r["victim_solo_ns"]
                                                                         for r in runs), 3),
                                 "blocked": sum(r["blocked"] for r in runs)}
    return {
        "experiment": "fp64", "paper": "Sec. 4.4.3 Table 3 (H100: util 24/48/69/91 %, speedup 1.93/1.87/1.33/1.03)",
        "gemm_4096_beside_fp64": beside,
        "kernel": "fp64 multiply chains (__dmul_rn), one 128-thread block per SM, 8 rounds of 1024 multiplies",
        "fp64_peak_dmul_per_s": fp64_peak,
        "fp64_peak_per_sm_per_clock": round(fp64_peak / (S * clk), 3),
        "scenarios": rows,
    }


def exp_l2(ctx, repeats, green=False):
    S = ctx.info["num_sms"]
    half = S // 2
    ids_a, ids_b = list(range(half)), list(range(half, S))
    if green:
        part = ctx.partition(half, fine=True)
        n_a, n_b = part["stressor_sms"], part["victim_sms"]  # A runs on the stressor side
    try:
        return _l2_sizes(ctx, repeats, S, half, ids_a, ids_b, (n_a, n_b) if green else None)
    finally:
        if green:
            ctx.partition_release()


def _l2_sizes(ctx, repeats, S, half, ids_a, ids_b, green):
    sizes_mib = [1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256]
    top = sizes_mib[-1] * MiB
    buf_a = I.torch_u32_as_i32(21, top // 4, "cuda")
    buf_b = I.torch_u32_as_i32(22, top // 4, "cuda")
    out = []
    for mib in sizes_mib:
        nb = mib * MiB
        per_round = half * P.STREAM_CHUNKS_PER_ROUND * 64 * 1024  # bytes of `half` 1024-thread blocks per round
        rounds = max(256, math.ceil(8 * nb / per_round))
        if green:
            a = stressor_cfg(A.IFR_S_L2, sm_count=green[0], blocks_per_sm=1, block=1024, buf=buf_a,
                             working_set_bytes=nb, seed=1, max_rounds=rounds, mask_mode=1)
            b = stressor_cfg(A.IFR_S_L2, sm_count=green[1], blocks_per_sm=1, block=1024, buf=buf_b,
                             working_set_bytes=nb, seed=2, max_rounds=rounds, mask_mode=1)
        else:
            a = with_mask(stressor_cfg(A.IFR_S_L2, blocks_per_sm=1, block=1024, buf=buf_a, working_set_bytes=nb,
                                       seed=1, max_rounds=rounds), ids_a)
            b = with_mask(stressor_cfg(A.IFR_S_L2, blocks_per_sm=1, block=1024, buf=buf_b, working_set_bytes=nb,
                                       seed=2, max_rounds=rounds), ids_b)
        pr = run_pair(ctx, a, b, repeats)
        bytes_a = half * rounds * P.STREAM_CHUNKS_PER_ROUND * 64 * 1024
        out.append({"mib_per_instance": mib, "rounds": rounds, "slowdown_a": round(pr["slowdown_a"], 3),
                    "slowdown_b": round(pr["slowdown_b"], 3),
                    "solo_a_gbs": round(bytes_a / (pr["solo_a_us"] * 1e3), 1),
                    "co_a_gbs": round(bytes_a / (pr["co_a_us"] * 1e3), 1), "ok": pr["all_ok"],
                    "overlapped": pr["all_overlapped"]})
    return {
        "experiment": "l2_green" if green else "l2", "paper": "Sec. 4.3 Fig. 3 (H100, 50 MB L2: no slowdown <= 8 MB, peak 2.15x at 16 MB, "
                                     "~1.12x beyond 26 MB)",
        "kernels": ("stream read (XOR fold) of its own set, one 1024-thread block per SM; " +
                    ("instances A and B in two green-context partitions of %d and %d SMs (mask_mode 1)" % green
                     if green else "instance A on SM ids 0..%d, B on %d..%d (disjoint, mask_mode 2)"
                     % (half - 1, half, S - 1))),
        "l2_bytes": ctx.info["l2_bytes"], "sizes": out,
    }


def exp_smem(ctx, repeats):
    S = ctx.info["num_sms"]
    victims, keep = [], []
    for dim, k in ((1024, 64), (2048, 16), (4096, 4)):
        a = I.torch_normal_bf16(31, dim * dim, "cuda").view(dim, dim)
        b = I.torch_normal_bf16(32, dim * dim, "cuda").view(dim, dim)
        c = torch.empty(dim, dim, device="cuda")
        keep += [a, b, c]
        victims.append(("gemm %d^3" % dim, victim_cfg(A.IFR_V_GEMM, a, b, c, m=dim, n=dim, k=dim, repeats=k)))
    ways = [1, 2, 4, 8, 16, 32]
    row = [stressor_cfg(A.IFR_S_SMEM_32W, sm_count=S, blocks_per_sm=2, block=256, smem_ways=w, seed=7)
           for w in ways]
    cells = ctx.sweep([v for _, v in victims], [row], repeats=repeats, batched=False)
    sl = slowdowns_from_cells(cells, len(victims), len(row))
    return {
        "experiment": "smem", "paper": "Sec. 4.4.1 Fig. 4 (H100 torch.mm: 1.79x at dims 2048, 3.75x at dims 1024, "
                                       "32-way)",
        "stressor": "n-strided shared-memory ld/st, 2 blocks of 256 threads on every SM",
        "ways": ways,
        "victims": [{"victim": name, **s} for (name, _), s in zip(victims, sl)],
        "note": "slowdown[0] is the zero-SM stressor (harness only); slowdown[i] is n = ways[i-1]",
    }


def exp_hol(ctx, repeats):
    S = ctx.info["num_sms"]
    rounds, period = 100, 100_000  # 10 ms of sleep, as in the paper

    def sleep(smem):
        return stressor_cfg(A.IFR_S_SLEEP, sm_count=S, blocks_per_sm=1, block=128, period_ns=period,
                            max_rounds=rounds, working_set_bytes=smem, seed=1)

    keep = {}
    R = 8192
    keep["vA"] = I.torch_normal_bf16(13, R * R, "cuda").view(R, R)
    keep["vx"] = I.torch_normal_bf16(14, R, "cuda")
    keep["vy"] = torch.empty(R, device="cuda")
    keep["s1"] = I.torch_uniform_pm1(16, 16384 * 4096, "cuda").view(16384, 4096)
    keep["o1"] = torch.empty_like(keep["s1"])
    keep["s2"] = I.torch_uniform_pm1(17, 4096 * 16384, "cuda").view(4096, 16384)
    keep["o2"] = torch.empty_like(keep["s2"])
    keep["gA"] = I.torch_normal_bf16(11, 4096 * 4096, "cuda").view(4096, 4096)
    keep["gB"] = I.torch_normal_bf16(12, 4096 * 4096, "cuda").view(4096, 4096)
    keep["gC"] = torch.empty(4096, 4096, device="cuda")
    cases = [
        ("gemv 8192x8192", 0, victim_cfg(A.IFR_V_GEMV, keep["vA"], keep["vx"], keep["vy"], m=R, k=R, repeats=16)),
        ("softmax 16384x4096 (256-thread blocks)", 0,
         victim_cfg(A.IFR_V_SOFTMAX, keep["s1"], None, keep["o1"], m=16384, n=4096, repeats=4)),
        ("softmax 4096x16384 (1024-thread blocks)", 0,
         victim_cfg(A.IFR_V_SOFTMAX, keep["s2"], None, keep["o2"], m=4096, n=16384, repeats=4)),
        ("gemm 4096^3, sleep blocks hold no shared memory", 0,
         victim_cfg(A.IFR_V_GEMM, keep["gA"], keep["gB"], keep["gC"], m=4096, n=4096, k=4096, repeats=4)),
        ("gemm 4096^3, sleep blocks hold 96 KiB of shared memory", 96 * 1024,
         victim_cfg(A.IFR_V_GEMM, keep["gA"], keep["gB"], keep["gC"], m=4096, n=4096, k=4096, repeats=4)),
    ]
    out = []
    for name, smem, v in cases:
        prof = ctx.victim_profile(v)
        runs = [ctx.colocate(sleep(smem), v) for _ in range(repeats)]
        med = lambda k: statistics.median(r[k] for r in runs)
        out.append({
            "victim": name, "block": prof["block"], "regs_per_thread": prof["regs_per_thread"],
            "smem_per_block": prof["static_smem"] + prof["dynamic_smem"], "sleep_smem": smem,
            "alone_us": round(med("victim_solo_ns") / 1e3, 1), "beside_sleep_us": round(med("victim_co_ns") / 1e3, 1),
            "latency_ratio": round(med("victim_co_ns") / med("victim_solo_ns"), 3),
            "blocked": sum(r["blocked"] for r in runs), "runs": len(runs),
            "sleep_us": round(med("stress_co_ns") / 1e3, 1), "ok": all(r["status"] == A.IFR_OK for r in runs)})
    sp = ctx.stressor_profile(sleep(0))
    return {
        "experiment": "hol", "paper": "Sec. 4.2 (H100: Llama3-8B decode TBT 7.53 -> 16.56 ms beside a 10 ms sleep "
                                      "kernel; a 64512-register block cannot join a 2048-register sleep block)",
        "sleep_kernel": "one 128-thread block per SM, %d registers per thread, %d x %d us" % (
            sp["regs_per_thread"], rounds, period // 1000),
        "victims": out,
    }


def exp_bandwidth(ctx, repeats, hbm_buf):
    S = ctx.info["num_sms"]
    info = ctx.partition(S // 2, fine=True)
    try:
        nv, ns = info["victim_sms"], info["stressor_sms"]
        victims, _keep = _decode_victims()
        # 512-thread blocks: up to three fit per SM at the stream kernel's 40 registers
        # (two 1024-thread blocks would need 81 920 registers and never co-reside)
        levels = [(max(1, ns // 2), 1), (ns, 1), (ns, 2), (ns, 3)]
        row = [stressor_cfg(A.IFR_S_HBM, sm_count=n, blocks_per_sm=b, block=512, buf=hbm_buf,
                            working_set_bytes=hbm_buf.numel() * 4, seed=1, mask_mode=1) for n, b in levels]
        peak = P.measured_peaks()[0]["hbm_gbs"]
        bw = []
        for c in row:
            rate, _ = P.solo_rate(ctx, c, rounds=64)
            bw.append(round(rate / 1e9, 1))
        cells = ctx.sweep([v for _, v in victims], [row], repeats=repeats, batched=False)
        sl = slowdowns_from_cells(cells, len(victims), len(row))
        touched = max(c.timing.sms_touched for c in cells)
    finally:
        ctx.partition_release()
    return {
        "experiment": "bandwidth",
        "paper": "Sec. 4.3 Table 1 (H100 green contexts, 64 + 68 SMs: copy L2 util 37/68/87/95 %, memory "
                 "bandwidth util 27/51/69/81 % at 34/68/102/136 blocks; decode TBT up to 1.3x)",
        "partition": {"victim_sms": nv, "stressor_sms": ns, "victim_sms_touched_max": touched},
        "copy_blocks_of_512": [n * b for n, b in levels], "copy_gbs": bw,
        "copy_frac_of_hbm_peak": [round(x / peak, 3) for x in bw],
        "victims": [{"victim": name, **s} for (name, _), s in zip(victims, sl)],
        "note": "slowdown[0] is the zero-SM stressor (harness only); slowdown[i] is copy level i",
    }


def exp_variants(ctx, repeats, hbm_buf):
    S = ctx.info["num_sms"]
    G = 4096
    gA = I.torch_normal_bf16(11, G * G, "cuda").view(G, G)
    gB = I.torch_normal_bf16(12, G * G, "cuda").view(G, G)
    gC = torch.empty(G, G, device="cuda")
    victims = [victim_cfg(A.IFR_V_GEMM, gA, gB, gC, m=G, n=G, k=G, repeats=4, variant=v) for v in (0, 1)]
    kinds = [A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W, A.IFR_S_TENSOR, A.IFR_S_FMA, A.IFR_S_HBM]
    from . import workloads as W
    stressors = []
    for k in kinds:
        cfg = W.stressor_level_cfg(k, S, {"hbm": hbm_buf}, seed=3)
        t_cal = P.solo_rate(ctx, cfg)[1]["elapsed_ms"]
        rounds = max(1, round(P.CAL_ROUNDS[k] * 8.0 / max(t_cal, 1e-3)))  # about 8 ms of fixed work
        stressors.append((A.STRESSOR_NAMES[k], P.copy_cfg(cfg, max_rounds=rounds)))
    rows = []
    for v in victims:
        prof = ctx.victim_profile(v)
        solo = ctx.victim_launch(_with_repeats(v, 20))
        tf = 2.0 * G ** 3 * 20 / (solo["event_ms"] * 1e-3) / 1e12
        beside = {}
        for name, sc in stressors:
            runs = [ctx.colocate(sc, v) for _ in range(repeats)]
            ratio = statistics.median(r["victim_co_ns"] / r["victim_solo_ns"] for r in runs)
            beside[name] = {"latency_ratio": round(ratio, 3), "blocked": sum(r["blocked"] for r in runs),
                            "runs": len(runs)}
        rows.append({"variant": v.variant, "stages": 3 + v.variant,
                     "smem_per_block": prof["dynamic_smem"],
                     "regs_per_thread": prof["regs_per_thread"], "solo_tflops": round(tf, 1), "beside": beside})
    return {
        "experiment": "variants", "paper": "Sec. 5.3 (colocation-friendly kernel variants trade single-kernel "
                                           "speed for the chance to share an SM)",
        "victim": "BF16 GEMM %d^3, 4 launches per measurement" % G,
        "stressors": "full SMs, configuration-2 shapes, about 8 ms of fixed work", "variants": rows,
    }


def _with_repeats(v, repeats):
    """Copy of a victim configuration with another launch count."""
    c = victim_cfg(v.kind)
    for name, _ in v._fields_:
        setattr(c, name, getattr(v, name))
    c.repeats = repeats
    return c


def _step(kernels, cells, row_len):
    """Per-kernel slowdown rows and the decode step latency (us) at each level."""
    per = lambda t: (t.t_end_ns - t.t_start_ns) / max(1, t.repeats)
    sl = slowdowns_from_cells(cells, len(kernels), row_len)
    step = []
    for lv in range(row_len + 1):
        tot = 0.0
        for v, s in enumerate(sl):
            x = s["slowdown"][lv]
            tot += s["solo_us"] * (x if x is not None else float("nan"))
        step.append(round(tot, 1))
    return sl, step


def exp_decode(ctx, repeats, hbm_buf):
    from . import colocate_config5 as C5
    S = ctx.info["num_sms"]
    clk = ctx.info["sm_clock_khz"] * 1e3
    kern, _keep = C5.decoder_kernels(S, "cuda", phases=("decode",))
    names = sorted(kern)
    victims = [kern[n] for n in names]
    for v in victims:
        C5.set_launches(ctx, v)
    # (a) compute kernel S1..S4 on the same SMs (Table 2, Fig. 5)
    ilps = [1, 2, 4, 8]
    row = [stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=1, block=128, ilp=i, seed=4) for i in ilps]
    ipc = [round(issue_rate(P.solo_rate(ctx, c, rounds=32)[0] / 2, S, clk), 3) for c in row]
    cells = ctx.sweep(victims, [row], repeats=repeats, batched=False)
    sl_a, step_a = _step(victims, cells, len(row))
    # (b) the copy kernel in the other green-context partition (Table 1)
    part = ctx.partition(S // 2, fine=True)
    try:
        ns = part["stressor_sms"]
        levels = [(max(1, ns // 2), 1), (ns, 1), (ns, 2), (ns, 3)]
        row_b = [stressor_cfg(A.IFR_S_HBM, sm_count=n, blocks_per_sm=b, block=512, buf=hbm_buf,
                              working_set_bytes=hbm_buf.numel() * 4, seed=1, mask_mode=1) for n, b in levels]
        for v in victims:
            C5.set_launches(ctx, v)  # alone on the victim partition
        cells_b = ctx.sweep(victims, [row_b], repeats=repeats, batched=False)
        sl_b, step_b = _step(victims, cells_b, len(row_b))
    finally:
        ctx.partition_release()
    return {
        "experiment": "decode",
        "paper": "Table 2 (RTX3090 Gemma3-1B TBT 5.59 / 5.75 / 6.00 / 6.24 / 10.74 ms for S0-S4), Table 1 (H100 "
                 "Llama3.1-8B decode up to 1.3x beside a copy in another green context), Fig. 5 (per-kernel)",
        "kernels": names,
        "compute": {"scenarios": ["S0"] + ["S%d (ILP %d)" % (i + 1, x) for i, x in enumerate(ilps)],
                    "compute_issue_rate": [0.0] + ipc, "step_us": step_a,
                    "per_kernel": {n: s for n, s in zip(names, sl_a)}},
        "copy_partition": {"partition": part, "copy_blocks_of_512": [n * b for n, b in levels], "step_us": step_b,
                           "per_kernel": {n: s for n, s in zip(names, sl_b)}},
        "note": "step_us[0] is the zero-SM stressor level (harness only, = the kernels alone)",
    }


NAMES = ["pitfall1", "pitfall2", "ipc", "fp64", "l2", "l2_green", "smem", "hol", "bandwidth", "variants", "decode"]


def main(argv=None):
    import paper_2501_16909_b300 as ifr

    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=NAMES)
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    bad = [n for n in a.names if n not in NAMES]
    if bad:
        raise SystemExit("unknown experiment(s) %s; choose from %s" % (bad, NAMES))
    ctx = ifr.Context(0)
    results = []
    pk = None
    hbm = None
    for name in a.names:
        t0 = time.perf_counter()
        if name == "pitfall1":
            r = exp_pitfall1(ctx, a.repeats)
        elif name == "pitfall2":
            hbm = hbm if hbm is not None else I.torch_u32_as_i32(1, (4 * GiB) // 4, "cuda")
            r = exp_pitfall2(ctx, a.repeats, hbm)
        elif name == "ipc":
            r = exp_ipc(ctx, a.repeats)
        elif name == "fp64":
            pk = pk or P.peaks(ctx)
            r = exp_fp64(ctx, a.repeats, pk[A.IFR_S_FP64][0])
        elif name == "l2":
            r = exp_l2(ctx, a.repeats)
        elif name == "l2_green":
            r = exp_l2(ctx, a.repeats, green=True)
        elif name == "hol":
            r = exp_hol(ctx, a.repeats)
        elif name == "decode":
            hbm = hbm if hbm is not None else I.torch_u32_as_i32(1, (4 * GiB) // 4, "cuda")
            r = exp_decode(ctx, a.repeats, hbm)
        elif name == "variants":
            hbm = hbm if hbm is not None else I.torch_u32_as_i32(1, (4 * GiB) // 4, "cuda")
            r = exp_variants(ctx, a.repeats, hbm)
        elif name == "bandwidth":
            hbm = hbm if hbm is not None else I.torch_u32_as_i32(1, (4 * GiB) // 4, "cuda")
            r = exp_bandwidth(ctx, a.repeats, hbm)
        else:
            r = exp_smem(ctx, a.repeats)
        r["seconds"] = round(time.perf_counter() - t0, 2)
        results.append(r)
        print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(results, f, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
