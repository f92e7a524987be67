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
            baseline's sensitivity curves (measured on base kinds only) never saw;
  kind      leave one stressor kind out: trained without any co-runner of that
            kind (base rows and variants), tested on them; pooled over the kinds.
Features are measured solo quantities of both sides (see the predictor module):
no configuration knob (ILP, conflict degree, duty) is an input.
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


def set_launches(ctx, cfg, target_ns=50000.0, cap=64):
    """K back-to-back launches per measurement so that K launches span ~target_ns."""
    cfg.repeats = 1
    tm = ctx.victim_launch(cfg)
    one = max(1.0, float(tm["t_end_ns"] - tm["t_start_ns"]))
    cfg.repeats = int(max(1, min(cap, round(target_ns / one))))


def _beside(ctx, victims, level_rows, repeats=1):
    """Graph-batched sweep of `victims` beside every configuration of `level_rows`
    ([rows][levels]); returns {(victim, row, level 1..L): median slowdown}."""
    from paper_2501_16909_b300 import plan
    from paper_2501_16909_b300.sweep_config3 import slowdown_table

    windows = plan.solo_windows(ctx, victims)
    t_launch = plan.sched_launch_ns(ctx, level_rows)
    _, lv_b = plan.mode_levels(level_rows, windows, t_launch)
    cells = ctx.sweep(victims, lv_b, repeats, batched=True)
    sd, _ = slowdown_table(cells)
    return sd, cells


def collect(ctx, repeats=2, log=print, row_names=None):
    """Measure every (victim, co-runner) pair and both sides' solo features; returns a
    dict of numpy arrays.

    1. every co-runner row is autotuned (8 or 16 intensities);
    2. each tuned configuration runs alone once more (fixed work): its block logs
       give the SMs and blocks it held, its CUDA-event time its rate;
    3. its pressure: the six probe kernels run beside it (graph-batched);
    4. each victim's sensitivity: its slowdown beside every stressor kind at full
       intensity (a separate graph-batched sweep);
    5. the pairs: every victim beside every tuned configuration (graph-batched)."""
    import torch

    import ifr_inputs as I
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import autotune, peaks, predictor, workloads
    from paper_2501_16909_b300.sweep_config3 import slowdown_table

    S = ctx.info["num_sms"]
    bufs = {"l2": I.torch_u32_as_i32(3, (workloads.L2_SET_BYTES) // 4, "cuda"),
            "hbm": I.torch_u32_as_i32(1, (4 << 30) // 4, "cuda")}
    victims, vkinds, _t = workloads.config3_victims("cuda")
    probes, _pt = workloads.probe_victims(S, "cuda")
    for c in probes:
        set_launches(ctx, c)
    pk = peaks.peaks(ctx, bufs["l2"])
    rows = corunner_rows(S, bufs)
    if row_names is not None:  # a reduced collection: only these co-runner rows
        rows = [r for r in rows if r[0] in row_names]
    tuned = []
    t0 = time.perf_counter()
    for name, k, base, fr in rows:
        tuner = autotune.Tuner(ctx, base, pk[k][0])
        _, lv = tuner.tune(fr)
        cfgs = [peaks.copy_cfg(base, sm_count=l.sm_count, duty=(l.duty if l.duty < 1 else 0.0)) for l in lv]
        tuned.append((name, k, cfgs, [l.frac_of_peak for l in lv], [l.rate for l in lv]))
    log("autotuned %d rows in %.1f s" % (len(rows), time.perf_counter() - t0))
    # 2. solo runs of every tuned configuration (block logs: SMs used, active blocks)
    solo = {}
    for r, (_n, _k, cfgs, _f, _rt) in enumerate(tuned):
        for l, cfg in enumerate(cfgs):
            _rate, res = peaks.solo_rate(ctx, cfg)
            solo[(r, l)] = res
    # 3. pressure of every tuned configuration on the probes
    pres = {}
    t0 = time.perf_counter()
    for c0 in range(0, len(tuned), 16):
        chunk = tuned[c0:c0 + 16]
        sd, _ = _beside(ctx, probes, [cfgs for _, _, cfgs, _, _ in chunk])
        for r in range(len(chunk)):
            for l in range(len(chunk[r][2])):
                pres[(c0 + r, l)] = [sd.get((p, r, l + 1), float("nan")) for p in range(len(probes))]
    log("probe pressure of %d configurations in %.1f s" % (len(pres), time.perf_counter() - t0))
    # 4. victims' sensitivity to every stressor kind at full intensity
    full = workloads.config3_base_stressors(S, bufs, predictor.SENSITIVITY_KINDS)
    sd_full, _ = _beside(ctx, victims, [[c] for c in full])
    sens = [[sd_full.get((v, r, 1), float("nan")) for r in range(len(full))] for v in range(len(victims))]
    # 5. the pairs
    vprof = [ctx.victim_profile(v) for v in victims]
    X_v, X_c, y, meta = [], [], [], []
    for c0 in range(0, len(tuned), 16):
        chunk = tuned[c0:c0 + 16]
        t1 = time.perf_counter()
        sd, cells = _beside(ctx, victims, [cfgs for _, _, cfgs, _, _ in chunk], repeats)
        log("sweep rows %d..%d: %d cells, %d valid, %.1f s" % (c0, c0 + len(chunk) - 1, len(cells),
                                                               sum(c.valid for c in cells), time.perf_counter() - t1))
        _, t0v = slowdown_table(cells)
        sms = {}
        for c in cells:
            if c.stressor < 0 and c.valid:
                sms[c.victim] = max(sms.get(c.victim, 0), c.timing.sms_touched)
        fv = {v: predictor.victim_features(vprof[v], t0v[v], sms.get(v, S), sens[v], pk, S) for v in t0v}
        for r, (name, k, cfgs, fracs, rates) in enumerate(chunk):
            for l, (cfg, frac, rate) in enumerate(zip(cfgs, fracs, rates)):
                prof = ctx.stressor_profile(cfg)
                fc = predictor.stressor_corunner_features(prof, cfg, rate, frac, pk, solo[(c0 + r, l)],
                                                          pres[(c0 + r, l)], S)
                for v in range(len(victims)):
                    key = (v, r, l + 1)
                    if key not in sd or v not in fv:
                        continue
                    X_v.append(fv[v])
                    X_c.append(fc)
                    y.append(sd[key])
                    meta.append((v, c0 + r, l, k, frac))
    torch.cuda.synchronize()
    m = np.array(meta, np.float64)
    return {"Xv": np.array(X_v), "Xc": np.array(X_c), "y": np.array(y), "victim": m[:, 0].astype(int),
            "row": m[:, 1].astype(int), "level": m[:, 2].astype(int), "kind": m[:, 3].astype(int), "frac": m[:, 4],
            "row_names": np.array([t[0] for t in tuned]),
            "n_base_rows": sum(1 for t in tuned if t[0].endswith("/a") or t[0].endswith("/b")),
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


SPLITS = ("random", "unseen", "kind")


def evaluate(ctx, d, split="random", seed=5, max_epochs=500, log=None):
    """MAPE of the MLP and of the baseline on held-out measured pairs.  Splits:
    random (20 % of all pairs), unseen (the pairs of 20 % of the variant
    configurations) and kind (leave one stressor kind out: for every kind, train on
    the pairs of the other kinds' co-runners, base rows and variants, and test on
    that kind's; the figures pool all seven folds)."""
    if split == "kind":
        res = [evaluate(ctx, d, ("kind", k), seed, max_epochs, log) for k in np.unique(d["kind"])]
        n = sum(r["test_pairs"] for r in res)
        pool = lambda key: round(sum(r[key] * r["test_pairs"] for r in res) / n, 4)  # noqa: E731
        return {"split": "kind", "train_pairs": int(np.mean([r["train_pairs"] for r in res])),
                "test_pairs": int(n), "epochs": int(sum(r["epochs"] for r in res)),
                "train_s": round(sum(r["train_s"] for r in res), 2), "mlp_mape": pool("mlp_mape"),
                "baseline_mape": pool("baseline_mape"),
                "mlp_mape_by_held_out_kind": {r["held_out"]: r["mlp_mape"] for r in res}}
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import predictor as PR

    n = len(d["y"])
    rng = np.random.default_rng(seed)
    base = d["row"] < d["n_base_rows"]
    held_kind = None
    if split == "random":
        test = np.zeros(n, bool)
        test[rng.permutation(n)[: n // 5]] = True
    elif split == "unseen":
        cfg_id = d["row"] * 100 + d["level"]
        var_ids = np.unique(cfg_id[~base])
        held = rng.permutation(var_ids)[: max(1, len(var_ids) // 5)]
        test = np.isin(cfg_id, held)
    else:
        held_kind = int(split[1])
        test = d["kind"] == held_kind
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
    return {"split": split if held_kind is None else "kind", "train_pairs": int(len(fit_idx)), "val_pairs": int(nv),
            "test_pairs": int(len(te)),
            "held_out": A.STRESSOR_NAMES[held_kind] if held_kind is not None else None,
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
    for split in SPLITS:
        out[split] = evaluate(ctx, d, split, max_epochs=a.max_epochs)
    ctx.close()
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
