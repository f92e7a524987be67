"""Configuration 5: colocate two synthetic decoder-layer kernel streams and score
every kernel pair with the slowdown predictor.

    python -m paper_2501_16909_b300.colocate_config5 [--repeats R] [--save out.npz]

The paper's setting (Sec. 4: LLM decode colocated with other work) with its
workloads replaced by synthetic kernels of a decoder layer (hidden 4096, 32 heads
of 128, FFN 11008, BF16 operands):

  prefill (batch 8 x 2048 tokens = 16384 rows): layernorm, QKV GEMM 16384x12288x4096,
    one head's QK^T GEMM 2048x2048x128, row softmax over all 256 heads' scores
    (524288 x 2048), one head's PV GEMM 2048x128x2048, O-projection
    16384x4096x4096, gate/up GEMM 16384x11008x4096, SiLU-mul (triad-shaped
    elementwise, 16384 x 11008), down GEMM 16384x4096x11008;
  decode (batch 64, KV length 4096): layernorm 64x4096, QKV 128x12288x4096 (the
    batch padded to the GEMM's 128-row tile), q.K^T as a GEMV over the whole K
    cache (64x32x4096 rows of 128), softmax 2048x4096, P.V as a GEMV over the V
    cache (64x32x128 rows of 4096), O-projection 128x4096x4096, gate/up
    128x11008x4096, SiLU-mul 64x11008, down 128x4096x11008.

Every ordered pair (decode victim, prefill co-runner) and (prefill victim,
decode co-runner) is measured with ifr_corun (median of R repeats).  The
predictor is trained on the configuration-4 stressor pairs plus kernel-with-
kernel pairs among the configuration-3 victims, then scores the configuration-5
pairs it never saw; the baseline is the per-resource estimator
1 + max_r S_v,r(x_c,r) over the victim's measured sensitivity curves (a stressor
sweep of each configuration-5 kernel) and the co-runner's solo resource fractions.
Both sides' features are measured (predictor module): a kernel's sensitivity is its
slowdown beside each stressor kind at full intensity, a co-runner kernel's pressure
the slowdown of six probe kernels beside it (ifr_corun).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def decoder_kernels(num_sms, device="cuda", phases=("prefill", "decode")):
    """{name: ifr_victim_cfg} for the prefill and / or decode kernel lists, plus the
    tensors.  Memory-bound kernels use 4 blocks of 256 threads per SM (half the SM's
    threads) so that a partner kernel can be resident beside them."""
    import torch

    import ifr_inputs as I
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import victim_cfg

    t = {}
    seed = [200]

    def nb(n):
        seed[0] += 1
        return I.torch_normal_bf16(seed[0], n, device)

    def un(n):
        seed[0] += 1
        return I.torch_uniform_pm1(seed[0], n, device)

    def gemm(M, N, K):
        a, b, c = nb(M * K).view(M, K), nb(N * K).view(N, K), torch.empty(M, N, device=device)
        t[len(t)] = (a, b, c)
        return victim_cfg(A.IFR_V_GEMM, a, b, c, m=M, n=N, k=K)

    def gemv(R, W):
        a, x, y = nb(R * W).view(R, W), nb(W), torch.empty(R, device=device)
        t[len(t)] = (a, x, y)
        return victim_cfg(A.IFR_V_GEMV, a, x, y, m=R, k=W, grid=4 * num_sms)

    def rows(kind, R, W):
        x = un(R * W).view(R, W)
        y = torch.empty_like(x)
        t[len(t)] = (x, y)
        return victim_cfg(kind, x, None, y, m=R, n=W, grid=4 * num_sms)

    def triad(n):
        b, c, a = un(n), un(n), torch.empty(n, device=device)
        t[len(t)] = (a, b, c)
        return victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=1.0, grid=4 * num_sms)

    T, H, F = 16384, 4096, 11008
    k = {}
    if "prefill" in phases:
        k.update(_prefill(gemm, rows, triad, T, H, F, A))
    if "decode" in phases:
        k.update(_decode(gemm, gemv, rows, triad, H, F, A))
    return k, t


def _prefill(gemm, rows, triad, T, H, F, A):
    return {
        "prefill.layernorm": rows(A.IFR_V_LAYERNORM, T, H),
        "prefill.qkv": gemm(T, 3 * H, H),
        "prefill.qk_head": gemm(2048, 2048, 128),
        "prefill.softmax": rows(A.IFR_V_SOFTMAX, 8 * 32 * 2048, 2048),
        "prefill.pv_head": gemm(2048, 128, 2048),
        "prefill.oproj": gemm(T, H, H),
        "prefill.gate_up": gemm(T, F, H),
        "prefill.silu_mul": triad(T * F),
        "prefill.down": gemm(T, H, F),
    }


def _decode(gemm, gemv, rows, triad, H, F, A):
    return {
        "decode.layernorm": rows(A.IFR_V_LAYERNORM, 64, H),
        "decode.qkv": gemm(128, 3 * H, H),
        "decode.qk": gemv(64 * 32 * 4096, 128),
        "decode.softmax": rows(A.IFR_V_SOFTMAX, 64 * 32, 4096),
        "decode.pv": gemv(64 * 32 * 128, 4096),
        "decode.oproj": gemm(128, H, H),
        "decode.gate_up": gemm(128, F, H),
        "decode.silu_mul": triad(64 * F),
        "decode.down": gemm(128, H, F),
    }


def set_launches(ctx, cfg, target_ns=100000.0, cap=256):
    """K so that K launches span about target_ns (at least 1)."""
    cfg.repeats = 1
    tm = ctx.victim_launch(cfg)
    one = max(1.0, float(tm["t_end_ns"] - tm["t_start_ns"]))
    cfg.repeats = int(max(1, min(cap, math.ceil(target_ns / one))))
    return one


def kernel_pairs(ctx, victims, corunners, repeats=3, blocked=None):
    """Median victim slowdown of every (victim, co-runner) pair via ifr_corun; pairs
    whose victim could not be co-resident (head-of-line blocked) go to `blocked`."""
    out = {}
    for i, v in enumerate(victims):
        for j, c in enumerate(corunners):
            sd, nb = [], 0
            for _ in range(repeats):
                r = ctx.corun(v, c)
                if r["valid"]:
                    sd.append(r["victim_slowdown"])
                elif r["blocked"]:
                    nb += 1
            if sd:
                out[(i, j)] = statistics.median(sd)
            elif nb and blocked is not None:
                blocked.append((i, j))
    return out


def half_occupancy(cfg, num_sms):
    """Copy of a memory-bound victim configuration with 4 blocks per SM."""
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import victim_cfg

    c = victim_cfg(cfg.kind)
    for name, _ in cfg._fields_:
        setattr(c, name, getattr(cfg, name))
    if cfg.kind != A.IFR_V_GEMM:
        c.grid = 4 * num_sms
    return c


def solo_facts(ctx, cfgs):
    """Solo time per launch (ns) and SMs touched of every kernel configuration."""
    ns, sms = [], []
    for c in cfgs:
        K = c.repeats
        c.repeats = 1
        tm = ctx.victim_launch(c)
        c.repeats = K
        ns.append(float(tm["t_end_ns"] - tm["t_start_ns"]))
        sms.append(tm["sms_touched"])
    return ns, sms


def probe_pressure(ctx, kernels, probes):
    """Slowdown of each probe kernel beside each kernel (ifr_corun, the kernel as the
    co-runner chain); NaN where the probe could not run beside it."""
    out = []
    for c in kernels:
        row = []
        for p in probes:
            r = ctx.corun(p, c)
            row.append(r["victim_slowdown"] if r["valid"] else float("nan"))
        out.append(row)
    return out


def full_sensitivity(ctx, cfgs, bufs):
    """Slowdown of every kernel beside each stressor kind at full intensity."""
    from paper_2501_16909_b300 import predictor as PR
    from paper_2501_16909_b300 import train_predictor as TP
    from paper_2501_16909_b300 import workloads

    full = workloads.config3_base_stressors(ctx.info["num_sms"], bufs, PR.SENSITIVITY_KINDS)
    sd, _ = TP._beside(ctx, cfgs, [[c] for c in full], repeats=2)
    return [[sd.get((v, r, 1), float("nan")) for r in range(len(full))] for v in range(len(cfgs))]


def features_of(ctx, cfgs, pk, sens, pressure):
    """(victim features, co-runner features, solo ns) of kernel configurations."""
    from paper_2501_16909_b300 import predictor as PR

    S = ctx.info["num_sms"]
    ns, sms = solo_facts(ctx, cfgs)
    fv, fc = [], []
    for i, c in enumerate(cfgs):
        prof = ctx.victim_profile(c)
        fv.append(PR.victim_features(prof, ns[i], sms[i], sens[i], pk, S))
        fc.append(PR.kernel_corunner_features(prof, ns[i], sms[i], pressure[i], pk, S))
    return np.array(fv), np.array(fc), ns


def main(argv=None):
    import torch

    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import train_predictor as TP

    ap = argparse.ArgumentParser()
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--pairs-npz", default=None, help="configuration-4 pairs saved by train_predictor --save")
    ap.add_argument("--save", default=None)
    ap.add_argument("--members", type=int, default=5, help="MLPs in the predictor ensemble")
    ap.add_argument("--max-epochs", type=int, default=500)
    ap.add_argument("--kernels", default=None,
                    help="comma-separated kernel names: score only the pairs among these (a reduced run)")
    ap.add_argument("--rows", default=None,
                    help="comma-separated co-runner rows of the training collection (a reduced run)")
    ap.add_argument("--co-idx", default=None, help="comma-separated configuration-3 co-runner indices")
    ap.add_argument("--occupancy-csv", default=None,
                    help="ncu achieved-occupancy capture of the kernels (profile_case config5_kernels): "
                         "adds the Usher / Orion pairing rules' scores")
    a = ap.parse_args(argv)
    log = lambda *x: print(*x, file=sys.stderr)  # noqa: E731
    ctx = ifr.Context(0)
    # 1. training data: stressor pairs (configuration 4) + kernel pairs among configuration-3 victims
    t0 = time.perf_counter()
    if a.pairs_npz and os.path.exists(a.pairs_npz):
        d = dict(np.load(a.pairs_npz, allow_pickle=True))
    else:
        d = TP.collect(ctx, repeats=2, log=log, row_names=a.rows.split(",") if a.rows else None)
    log("stressor pairs: %d (%.1f s)" % (len(d["y"]), time.perf_counter() - t0))
    out = score(ctx, d, repeats=a.repeats, members=a.members, max_epochs=a.max_epochs,
                kernels=a.kernels.split(",") if a.kernels else None,
                co_idx=[int(x) for x in a.co_idx.split(",")] if a.co_idx else None,
                occupancy_csv=a.occupancy_csv, save=a.save, log=log)
    ctx.close()
    torch.cuda.synchronize()
    print(json.dumps(out))
    return out


def score(ctx, d, repeats=3, members=5, max_epochs=500, kernels=None, co_idx=None, occupancy_csv=None, save=None,
          log=lambda *x: None):
    """Steps 2-3 on a context and the configuration-4 pairs `d` (train_predictor.collect):
    kernel pairs among configuration-3 victims, the configuration-5 pairs and their
    sensitivity curves, then the predictor ensemble against the measurements."""
    import paper_2501_16909_b300 as ifr  # noqa: F401
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import peaks, plan, predictor as PR, train_predictor as TP, workloads
    from paper_2501_16909_b300.sweep_config3 import slowdown_table

    S = ctx.info["num_sms"]
    import ifr_inputs as I

    l2 = I.torch_u32_as_i32(3, workloads.L2_SET_BYTES // 4, "cuda")
    bufs = {"l2": l2, "hbm": I.torch_u32_as_i32(1, (4 << 30) // 4, "cuda")}
    pk = peaks.peaks(ctx, l2)
    probes, _pt = workloads.probe_victims(S, "cuda")
    for c in probes:
        TP.set_launches(ctx, c)
    v3, v3k, _t3 = workloads.config3_victims("cuda")
    v3 = [half_occupancy(c, S) for c in v3]
    for c in v3:
        set_launches(ctx, c, 50000.0)
    if co_idx is None:
        co_idx = [0, 5, 10, 16, 21, 26, 32, 37, 42, 48, 53, 58]  # 3 GEMMs, 3 GEMVs, 3 softmax, 3 layernorm
    t0 = time.perf_counter()
    kp = kernel_pairs(ctx, v3, [v3[j] for j in co_idx], repeats=1)
    pres3 = [[float("nan")] * len(probes)] * len(v3)
    for j, pr in zip(co_idx, probe_pressure(ctx, [v3[j] for j in co_idx], probes)):
        pres3[j] = pr
    F3v, F3c, _ = features_of(ctx, v3, pk, full_sensitivity(ctx, v3, bufs), pres3)
    log("kernel pairs: %d (%.1f s)" % (len(kp), time.perf_counter() - t0))
    Xk = np.array([np.concatenate([F3v[i], F3c[co_idx[j]]]) for (i, j) in kp])
    yk = np.array(list(kp.values()))
    X = np.concatenate([np.concatenate([d["Xv"], d["Xc"]], axis=1), Xk])
    y = np.concatenate([d["y"], yk])

    # 2. configuration-5 kernels, their pairs and sensitivity curves
    kern, _t5 = decoder_kernels(S, "cuda")
    names = [n for n in kern if kernels is None or n in kernels]
    cfgs = [kern[n] for n in names]
    for c in cfgs:
        set_launches(ctx, c, 100000.0)
    F5v, F5c, solo5 = features_of(ctx, cfgs, pk, full_sensitivity(ctx, cfgs, bufs), probe_pressure(ctx, cfgs, probes))
    pre = [i for i, n in enumerate(names) if n.startswith("prefill")]
    dec = [i for i, n in enumerate(names) if n.startswith("decode")]
    t0 = time.perf_counter()
    blk_dp, blk_pd = [], []
    m_dp = kernel_pairs(ctx, [cfgs[i] for i in dec], [cfgs[j] for j in pre], repeats, blk_dp)
    m_pd = kernel_pairs(ctx, [cfgs[i] for i in pre], [cfgs[j] for j in dec], repeats, blk_pd)
    log("config-5 pairs: %d + %d (%.1f s)" % (len(m_dp), len(m_pd), time.perf_counter() - t0))
    pairs = [(dec[i], pre[j], s) for (i, j), s in m_dp.items()] + [(pre[i], dec[j], s) for (i, j), s in m_pd.items()]

    # victims' sensitivity curves: one batched stressor sweep (7 kinds x 8 autotuned levels)
    from paper_2501_16909_b300 import autotune

    base = workloads.config3_base_stressors(S, bufs)
    fr = [(l + 1) / 8 for l in range(8)]
    levels, report = autotune.tuned_levels(ctx, base, pk, fr)
    windows = plan.solo_windows(ctx, cfgs)
    _, lv_b = plan.mode_levels(levels, windows, plan.sched_launch_ns(ctx, levels))
    cells = ctx.sweep(cfgs, lv_b, 2, batched=True)
    sd, _ = slowdown_table(cells)
    curves = {}
    for r, rep in enumerate(report):
        xs = [0.0] + [l["frac_of_peak"] for l in rep["levels"]]
        for v in range(len(cfgs)):
            ss = [0.0] + [sd.get((v, r, l + 1), float("nan")) - 1.0 for l in range(8)]
            curves[(v, r)] = (np.array(xs), np.nan_to_num(np.array(ss), nan=0.0))
    kinds = [b.kind for b in base]
    slot = {A.IFR_S_HBM: 0, A.IFR_S_L2: 1, A.IFR_S_TENSOR: 2, A.IFR_S_FMA: 3, A.IFR_S_SMEM_CF: 4,
            A.IFR_S_SMEM_32W: 4, A.IFR_S_SCHED: 5}

    def baseline(v, c):
        best = 0.0
        for r, k in enumerate(kinds):
            if k == A.IFR_S_SMEM_32W:
                continue  # a kernel's shared-memory use is scored with the conflict-free curve
            x = F5c[c][slot[k]]
            xs, ss = curves[(v, r)]
            best = max(best, float(np.interp(x, xs, ss)))
        return 1.0 + best

    # 3. train on the training pairs, score configuration 5
    z = PR.Standardizer(X)
    rng = np.random.default_rng(5)
    idx = rng.permutation(len(y))
    nv = len(y) // 10
    # an ensemble of a.members MLPs: single models trained on these pairs scored the
    # configuration-5 pairs anywhere between 17 % and 27 % MAPE from run to run
    models = PR.train_ensemble(ctx, z(X[idx[nv:]]), y[idx[nv:]], z(X[idx[:nv]]), y[idx[:nv]], members=members,
                               max_epochs=max_epochs)
    Xt = np.array([np.concatenate([F5v[v], F5c[c]]) for v, c, _ in pairs])
    yt = np.array([s for _, _, s in pairs])
    pred = PR.predict_ensemble(models, z(Xt))
    single = PR.predict(models[0], z(Xt))
    base_pred = np.array([baseline(v, c) for v, c, _ in pairs])
    out = {
        "kernels": names, "solo_us": [round(s / 1e3, 2) for s in solo5], "launches": [c.repeats for c in cfgs],
        "training_pairs": int(len(y)), "kernel_training_pairs": int(len(yk)), "ensemble": len(models),
        "mlp_single_member_mape": round(PR.mape(single, yt), 4),
        "config5_pairs": len(pairs),
        "blocked_pairs": [(names[dec[i]], names[pre[j]]) for i, j in blk_dp] + [(names[pre[i]], names[dec[j]])
                                                                               for i, j in blk_pd],
        "measured_slowdown_median": round(float(np.median(yt)), 4),
        "measured_slowdown_max": round(float(np.max(yt)), 4),
        "mlp_mape": round(PR.mape(pred, yt), 4), "baseline_mape": round(PR.mape(base_pred, yt), 4),
        "mlp_mape_decode_victims": round(PR.mape(pred[: len(m_dp)], yt[: len(m_dp)]), 4),
        "mlp_mape_prefill_victims": round(PR.mape(pred[len(m_dp):], yt[len(m_dp):]), 4),
        "pairs": [{"victim": names[v], "corunner": names[c], "measured": round(s, 4), "mlp": round(float(p), 4),
                   "baseline": round(float(b), 4)} for (v, c, s), p, b in zip(pairs, pred, base_pred)],
        "kernel_info": {n: {"flops": prof["flops_per_launch"], "bytes": prof["bytes_per_launch"],
                            "uses_tensor": bool(prof["uses_tensor"])}
                        for n, prof in ((n, ctx.victim_profile(c)) for n, c in zip(names, cfgs))},
        "peaks": {"tensor": pk[A.IFR_S_TENSOR][0], "fp32": pk[A.IFR_S_FMA][0], "hbm": pk[A.IFR_S_HBM][0]},
    }
    if occupancy_csv:
        from paper_2501_16909_b300 import pairing

        with open(occupancy_csv) as f:
            occ = pairing.occupancy_by_kernel(names, pairing.parse_ncu_occupancy(f.read()))
        out["pairing"] = pairing.evaluate(out["pairs"], out["kernel_info"], occ, out["peaks"])
    if save:
        np.savez(save, X=X, y=y, Xt=Xt, yt=yt, pred=pred, base=base_pred)
    return out


if __name__ == "__main__":
    main()
