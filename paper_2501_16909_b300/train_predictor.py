"""Configuration 4: measure (victim, co-runner) pairs, train the slowdown predictor,
and compare it with the method without the network.

    python -m paper_2501_16909_b300.train_predictor [--repeats R] [--save data.npz]

Pairs: the 64 victims of configuration 3 against co-runner configurations —
the seven base stressor kinds at 16 autotuned intensities (fractions l/16 of their
full-SM rate, split into two rows of 8) and stressor variants at 8 autotuned
intensities (other ILP, bank-conflict degrees, footprints, scheduler block
lengths).  Every pair's slowdown is measured by the graph-batched sweep (median
over repeats of per-launch time over the median solo time).

Evaluations (seed 5):
  random    80/20 split over all pairs (the configuration's split);
  unseen    the MLP is trained on every base pair and 80 % of the variant
            configurations and tested on the pairs of the other 20 %, which the
            baseline's sensitivity curves (measured on base kinds only) never saw.
Baseline: 1 + S_v,r(x), the victim's measured slowdown-minus-one curve for the
base kind matching the co-runner's resource, at the co-runner's solo fraction x.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def corunner_rows(S, bufs):
    """[(name, base_kind, base_cfg, fractions)] — base kinds twice (odd / even
    sixteenths) and the variants (eighths)."""
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import workloads as W

    kinds = [A.IFR_S_SCHED, A.IFR_S_FMA, A.IFR_S_TENSOR, A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W, A.IFR_S_L2, A.IFR_S_HBM]
    odd = [(2 * i + 1) / 16 for i in range(8)]
    even = [(2 * i + 2) / 16 for i in range(8)]
    eighths = [(i + 1) / 8 for i in range(8)]
    rows = []
    for k in kinds:
        base = W.stressor_level_cfg(k, S, bufs, seed=k + 1)
        rows.append((A.STRESSOR_NAMES[k] + "/a", k, base, odd))
        rows.append((A.STRESSOR_NAMES[k] + "/b", k, base, even))
    var = [
        ("fma ilp1", A.IFR_S_FMA, dict(ilp=1)), ("fma ilp2", A.IFR_S_FMA, dict(ilp=2)),
        ("fma ilp4", A.IFR_S_FMA, dict(ilp=4)), ("fma b256 bps2", A.IFR_S_FMA, dict(block=256, blocks_per_sm=2)),
        ("smem ways2", A.IFR_S_SMEM_CF, dict(smem_ways=2)), ("smem ways4", A.IFR_S_SMEM_CF, dict(smem_ways=4)),
        ("smem ways8", A.IFR_S_SMEM_32W, dict(smem_ways=8)), ("smem ways16", A.IFR_S_SMEM_32W, dict(smem_ways=16)),
        ("smem cf bps1", A.IFR_S_SMEM_CF, dict(blocks_per_sm=1)),
        ("smem 32w bps1", A.IFR_S_SMEM_32W, dict(blocks_per_sm=1)),
        ("hbm bps1", A.IFR_S_HBM, dict(blocks_per_sm=1)), ("hbm b256", A.IFR_S_HBM, dict(block=256)),
        ("l2 bps1", A.IFR_S_L2, dict(blocks_per_sm=1)), ("l2 b1024 bps1", A.IFR_S_L2, dict(block=1024, blocks_per_sm=1)),
        ("tensor bps2", A.IFR_S_TENSOR, dict(blocks_per_sm=2)),
        ("sched 400cyc", A.IFR_S_SCHED, dict(sched_cycles=400)),
        ("sched 1600cyc", A.IFR_S_SCHED, dict(sched_cycles=1600)),
    ]
    for name, k, over in var:
        rows.append((name, k, W.stressor_level_cfg(k, S, bufs, seed=k + 1, **over), eighths))
    return rows


def collect(ctx, repeats=2, log=print):
    """Measure every (victim, co-runner) pair; returns a dict of numpy arrays."""
    import torch

    import ifr_inputs as I
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import autotune, peaks, plan, predictor, workloads
    from paper_2501_16909_b300.sweep_config3 import slowdown_table

    S = ctx.info["num_sms"]
    bufs = {"l2": I.torch_u32_as_i32(3, (workloads.L2_SET_BYTES) // 4, "cuda"), "hbm": I.torch_u32_as_i32(1, (4 << 30) // 4, "cuda")}
    victims, vkinds, _t = workloads.config3_victims("cuda")
    pk = peaks.peaks(ctx, bufs["l2"])
    rows = corunner_rows(S, bufs)
    tuned = []
    t0 = time.perf_counter()
    for name, k, base, fr in rows:
        tuner = autotune.Tuner(ctx, base, pk[k][0])
        _, lv = tuner.tune(fr)
        cfgs = [peaks.copy_cfg(base, sm_count=l.sm_count, duty=(l.duty if l.duty < 1 else 0.0)) for l in lv]
        tuned.append((name, k, cfgs, [l.frac_of_peak for l in lv]))
    log("autotuned %d rows in %.1f s" % (len(rows), time.perf_counter() - t0))
    vprof = [ctx.victim_profile(v) for v in victims]
    windows = plan.solo_windows(ctx, victims)
    X_v, X_c, y, meta = [], [], [], []
    for c0 in range(0, len(tuned), 16):
        chunk = tuned[c0:c0 + 16]
        levels = [cfgs for _, _, cfgs, _ in chunk]
        t_launch = plan.sched_launch_ns(ctx, levels)
        _, lv_b = plan.mode_levels(levels, windows, t_launch)
        t1 = time.perf_counter()
        cells = ctx.sweep(victims, lv_b, repeats, batched=True)
        log("sweep rows %d..%d: %d cells, %d valid, %.1f s" % (c0, c0 + len(chunk) - 1, len(cells),
                                                               sum(c.valid for c in cells), time.perf_counter() - t1))
        sd, t0v = slowdown_table(cells)
        for r, (name, k, cfgs, fracs) in enumerate(chunk):
            for l, (cfg, frac) in enumerate(zip(cfgs, fracs)):
                prof = ctx.stressor_profile(cfg)
                fc = predictor.stressor_features(prof, cfg, frac, S)
                for v in range(len(victims)):
                    key = (v, r, l + 1)
                    if key not in sd or v not in t0v:
                        continue
                    X_v.append(predictor.victim_features(vprof[v], t0v[v], pk, S))
                    X_c.append(fc)
                    y.append(sd[key])
                    meta.append((v, c0 + r, l, k, frac))
    torch.cuda.synchronize()
    m = np.array(meta, np.float64)
    return {"Xv": np.array(X_v), "Xc": np.array(X_c), "y": np.array(y), "victim": m[:, 0].astype(int),
            "row": m[:, 1].astype(int), "level": m[:, 2].astype(int), "kind": m[:, 3].astype(int), "frac": m[:, 4],
            "row_names": np.array([t[0] for t in tuned]), "n_base_rows": 14,
            "victim_kinds": np.array([A.VICTIM_NAMES[k] for k in vkinds])}


def sensitivity_curves(d, mask):
    """(victim, base kind) -> (x sorted, slowdown - 1) from the base rows in mask."""
    curves = {}
    for v in np.unique(d["victim"]):
        for k in np.unique(d["kind"]):
            sel = mask & (d["victim"] == v) & (d["kind"] == k) & (d["row"] < d["n_base_rows"])
            if not sel.any():
                continue
            xs = np.concatenate([[0.0], d["frac"][sel]])
            ss = np.concatenate([[0.0], d["y"][sel] - 1.0])
            o = np.argsort(xs)
            curves[(int(v), int(k))] = (xs[o], ss[o])
    return curves


def evaluate(ctx, d, split="random", seed=5, max_epochs=500, log=None):
    from paper_2501_16909_b300 import predictor as PR

    n = len(d["y"])
    rng = np.random.default_rng(seed)
    base = d["row"] < d["n_base_rows"]
    if split == "random":
        test = np.zeros(n, bool)
        test[rng.permutation(n)[: n // 5]] = True
    else:
        cfg_id = d["row"] * 100 + d["level"]
        var_ids = np.unique(cfg_id[~base])
        held = rng.permutation(var_ids)[: max(1, len(var_ids) // 5)]
        test = np.isin(cfg_id, held)
    train = ~test
    X = np.concatenate([d["Xv"], d["Xc"]], axis=1)
    # validation for early stopping: 10 % of the training pairs
    tr_idx = np.nonzero(train)[0]
    rng.shuffle(tr_idx)
    nv = max(1, len(tr_idx) // 10)
    va_idx, fit_idx = tr_idx[:nv], tr_idx[nv:]
    z = PR.Standardizer(X[fit_idx])
    model = PR.PredictorMLP(ctx)
    t0 = time.perf_counter()
    hist = PR.train(model, z(X[fit_idx]), d["y"][fit_idx], z(X[va_idx]), d["y"][va_idx], max_epochs=max_epochs,
                    log=log)
    train_s = time.perf_counter() - t0
    te = np.nonzero(test)[0]
    pred = PR.predict(model, z(X[te]))
    mlp_mape = PR.mape(pred, d["y"][te])
    # baseline curves from base rows of the training side (the 'unseen' split keeps all base rows)
    curves = sensitivity_curves(d, train | (split != "random"))
    bl = []
    for i in te:
        key = (int(d["victim"][i]), int(d["kind"][i]))
        bl.append(PR.baseline_predict(curves, *key, d["frac"][i]) if key in curves else 1.0)
    return {"split": split, "train_pairs": int(len(fit_idx)), "val_pairs": int(nv), "test_pairs": int(len(te)),
            "epochs": len(hist), "train_s": round(train_s, 2), "mlp_mape": round(mlp_mape, 4),
            "baseline_mape": round(PR.mape(bl, d["y"][te]), 4),
            "mlp_mape_by_victim_kind": {k: round(PR.mape(pred[d["victim_kinds"][d["victim"][te]] == k],
                                                         d["y"][te][d["victim_kinds"][d["victim"][te]] == k]), 4)
                                        for k in np.unique(d["victim_kinds"])}}


def main(argv=None):
    import paper_2501_16909_b300 as ifr

    ap = argparse.ArgumentParser()
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--save", default=None)
    ap.add_argument("--load", default=None)
    ap.add_argument("--max-epochs", type=int, default=500)
    a = ap.parse_args(argv)
    ctx = ifr.Context(0)
    if a.load:
        d = dict(np.load(a.load, allow_pickle=True))
        d["n_base_rows"] = int(d["n_base_rows"])
    else:
        d = collect(ctx, a.repeats, log=lambda *x: print(*x, file=sys.stderr))
        if a.save:
            np.savez(a.save, **d)
    out = {"pairs": int(len(d["y"])), "slowdown_median": round(float(np.median(d["y"])), 4),
           "slowdown_p90": round(float(np.quantile(d["y"], 0.9)), 4)}
    for split in ("random", "unseen"):
        out[split] = evaluate(ctx, d, split, max_epochs=a.max_epochs)
    ctx.close()
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
