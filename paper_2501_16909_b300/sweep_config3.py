"""Configuration 3: batched vs plain sweep over 64 uneven victims with autotuned levels.

    python -m paper_2501_16909_b300.sweep_config3 [--repeats R] [--levels L] [--out cells.jsonl]

1. builds the 64 victims of configuration 3 (seeded shapes, see
   workloads.config3_shapes) and the stressors' buffers;
2. autotunes, per stressor kind, the launch shape of each target intensity l/L of
   its full-intensity rate (autotune.Tuner, +-5 %);
3. runs the graph-batched sweep, the same with grouped persistent victims, and the
   plain launch-per-cell sweep on the same inputs and levels, timing each with the
   host clock around the ABI call;
4. reports cells/s of each, the fraction of valid cells, and how closely each
   batched mode agrees with the plain sweep on every (victim, stressor, level)
   slowdown;
5. optionally writes one JSON row per measured cell (raw timestamps included),
   the data the slowdown predictor is trained on.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def slowdown_table(cells):
    """{(victim, stressor, level): median per-launch time / median solo time}."""
    import paper_2501_16909_b300 as ifr

    rows = ifr.cells_to_dicts(cells)
    solo = {}
    for r in rows:
        if r["stressor"] < 0 and r["valid"]:
            solo.setdefault(r["victim"], []).append((r["t_end"] - r["t_start"]) / r["k"])
    t0 = {v: statistics.median(x) for v, x in solo.items()}
    acc = {}
    for r in rows:
        if r["stressor"] >= 0 and r["valid"] and r["victim"] in t0:
            acc.setdefault((r["victim"], r["stressor"], r["level"]), []).append((r["t_end"] - r["t_start"]) / r["k"])
    return {k: statistics.median(v) / t0[k[0]] for k, v in acc.items()}, t0


def main(argv=None):
    import torch

    import ifr_inputs as I
    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import autotune, peaks, plan, workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--levels", type=int, default=8)
    ap.add_argument("--out", default=None)
    ap.add_argument("--skip-plain", action="store_true")
    a = ap.parse_args(argv)

    ctx = ifr.Context(0)
    S = ctx.info["num_sms"]
    bufs = {"l2": I.torch_u32_as_i32(3, (workloads.L2_SET_BYTES) // 4, "cuda"), "hbm": I.torch_u32_as_i32(1, (4 << 30) // 4, "cuda")}
    victims, vkinds, tensors = workloads.config3_victims("cuda")
    pk = peaks.peaks(ctx, bufs["l2"])
    base = workloads.config3_base_stressors(S, bufs)
    fr = [(l + 1) / a.levels for l in range(a.levels)]
    t0 = time.perf_counter()
    levels, report = autotune.tuned_levels(ctx, base, pk, fr)
    tune_s = time.perf_counter() - t0
    windows = plan.solo_windows(ctx, victims)
    t_launch = plan.sched_launch_ns(ctx, levels)
    lv_plain, lv_batched = plan.mode_levels(levels, windows, t_launch)
    torch.cuda.synchronize()

    out = {"workload": "config3: 64 uneven victims x %d stressors x %d autotuned levels" % (len(base), a.levels),
           "repeats": a.repeats, "autotune_s": round(tune_s, 3),
           "autotune": [{"kind": r["kind"], "probes": r["probes"],
                         "levels": [(l["sm_count"], round(l["duty"], 3), round(l["frac_of_max"], 4)) for l in
                                    r["levels"]],
                         "max_err": round(max(abs(l["frac_of_max"] / l["target"] - 1) for l in r["levels"]), 4)}
                        for r in report]}
    # batched first (graph capture included in its time), then plain
    t0 = time.perf_counter()
    cb = ctx.sweep(victims, lv_batched, a.repeats, batched=True)
    tb = time.perf_counter() - t0
    out["batched"] = {"cells": len(cb), "seconds": round(tb, 3), "cells_per_s": round(len(cb) / tb, 1),
                      "valid": sum(c.valid for c in cb), "hol": sum(1 for c in cb if c.status == A.IFR_ERR_HOL)}
    sd_b, t0b = slowdown_table(cb)
    # the same graphs with grouped persistent victims
    t0 = time.perf_counter()
    cg = ctx.sweep(victims, lv_batched, a.repeats, batched=True, grouped=True)
    tg = time.perf_counter() - t0
    out["grouped"] = {"cells": len(cg), "seconds": round(tg, 3), "cells_per_s": round(len(cg) / tg, 1),
                      "valid": sum(c.valid for c in cg), "hol": sum(1 for c in cg if c.status == A.IFR_ERR_HOL)}
    sd_g, _ = slowdown_table(cg)
    if not a.skip_plain:
        t0 = time.perf_counter()
        cp = ctx.sweep(victims, lv_plain, a.repeats, batched=False)
        tp = time.perf_counter() - t0
        out["plain"] = {"cells": len(cp), "seconds": round(tp, 3), "cells_per_s": round(len(cp) / tp, 1),
                        "valid": sum(c.valid for c in cp), "hol": sum(1 for c in cp if c.status == A.IFR_ERR_HOL)}
        out["batched_over_plain"] = round(out["batched"]["cells_per_s"] / out["plain"]["cells_per_s"], 3)
        sd_p, _ = slowdown_table(cp)
        out["grouped_over_plain"] = round(out["grouped"]["cells_per_s"] / out["plain"]["cells_per_s"], 3)
        for name, sd in (("agreement", sd_b), ("agreement_grouped", sd_g)):
            common = [k for k in sd if k in sd_p]
            rel = sorted(abs(sd[k] / sd_p[k] - 1) for k in common)
            if rel:
                out[name] = {"pairs": len(rel), "median_rel_diff": round(rel[len(rel) // 2], 4),
                             "p90_rel_diff": round(rel[int(0.9 * (len(rel) - 1))], 4)}
                # per stressor kind: the median relative difference and the median of the
                # mode's slowdown over the plain sweep's (above 1: the mode measures more)
                per = {}
                for k in common:
                    per.setdefault(A.STRESSOR_NAMES[base[k[1]].kind], []).append(sd[k] / sd_p[k])
                out[name]["by_kind"] = {kk: {"median_rel_diff": round(statistics.median(abs(x - 1) for x in v), 4),
                                             "median_ratio": round(statistics.median(v), 4)}
                                        for kk, v in per.items()}
    if a.out:
        with open(a.out, "w") as f:
            for c in ifr.cells_to_dicts(cb):
                c["mode"] = "batched"
                c["victim_kind"] = A.VICTIM_NAMES[vkinds[c["victim"]]]
                f.write(json.dumps(c) + "\n")
    ctx.close()
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
