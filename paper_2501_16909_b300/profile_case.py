"""Run one stressor or victim alone, for profilers.

Profilers that replay kernels serialise them, so they cannot observe colocated
kernels (the paper makes the same point about NCU in Sec. 5.2).  This driver runs
one kernel kind in isolation on a small case so that a profiler can capture it:

    python -m paper_2501_16909_b300.profile_case <case> [--repeat N]

cases: hbm, l2 (--staging), fma, tensor, smem_cf, smem_32w, sched, fp64, sleep, gemm (--variant),
gemv, layernorm, softmax, hist, triad; gemm_variants, the solo throughput of every GEMM
variant at four shapes; config5_kernels, one launch of each configuration-5
decoder-layer kernel in order; and victim_bandwidth, which times every memory-bound
configuration-2 victim alone over grids of 0 (default), 1, 2, 4, 8 and 16 blocks per
SM (20 launches after a warm measurement; the GEMV also as variant 1, its rows
streamed into shared memory), then a triad moving the same bytes per launch, and
prints one JSON line per run; and
l2_set_sweep, which times the stream kernel on every SM (256 rounds per block) over
sets of 8..96 MiB for 2 x 512, 4 x 512 and 2 x 256 threads per SM; and stream_staging,
which times the HBM (4 GiB) and L2 (16 MiB) stressors with register loads and with TMA
bulk copies over four block shapes.  Inputs are the workloads' seeded inputs at the sizes
given below (the stream stressors use a 1 GiB / 48 MiB set; the victims use their
full configuration-2 shapes).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import ifr_inputs as I
    import paper_2501_16909_b300 as ifr
    from paper_2501_16909_b300 import _abi as A
    from paper_2501_16909_b300 import peaks as P
    from paper_2501_16909_b300 import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--sm-fraction", type=float, default=1.0)
    ap.add_argument("--variant", type=int, default=None,
                    help="GEMM variant (0-4) or GEMV variant (0, 1 = rows by bulk copies); default: the workload's")
    ap.add_argument("--block", type=int, default=None, help="stressors: threads per block")
    ap.add_argument("--bps", type=int, default=None, help="stressors: blocks per SM")
    ap.add_argument("--ilp", type=int, default=None, help="FMA / FP64 stressors: chains per thread")
    ap.add_argument("--staging", type=int, default=0,
                    help="L2 / HBM stressors: 0 = loads into registers, 1 = TMA bulk copies into shared memory")
    a = ap.parse_args(argv)
    ctx = ifr.Context(0)
    S = ctx.info["num_sms"]
    n_sm = max(1, round(a.sm_fraction * S))
    out = {"case": a.case, "sm_count": n_sm}
    stressors = {"hbm": A.IFR_S_HBM, "l2": A.IFR_S_L2, "fma": A.IFR_S_FMA, "tensor": A.IFR_S_TENSOR,
                 "smem_cf": A.IFR_S_SMEM_CF, "smem_32w": A.IFR_S_SMEM_32W, "sched": A.IFR_S_SCHED,
                 "fp64": A.IFR_S_FP64, "sleep": A.IFR_S_SLEEP}
    if a.case == "l2_set_sweep":
        buf = I.torch_u32_as_i32(3, (96 << 20) // 4, "cuda")
        for mib in (8, 16, 24, 32, 40, 48, 64, 96):
            for block, bps in ((512, 2), (512, 4), (256, 2)):
                cfg = ifr.stressor_cfg(A.IFR_S_L2, sm_count=S, blocks_per_sm=bps, block=block, buf=buf,
                                       working_set_bytes=mib << 20)
                rate, _res = P.solo_rate(ctx, cfg, rounds=256)
                print(json.dumps({"mib": mib, "block": block, "blocks_per_sm": bps, "gbs": round(rate / 1e9, 1)}))
        ctx.close()
        return
    if a.case == "stream_staging":
        # the stream stressor with register loads (staging 0) and with TMA bulk copies
        # (staging 1) on every SM: HBM over a 4 GiB set (64 rounds per block) and L2 over
        # the 16 MiB set (256 rounds), 2 or 4 blocks of 512 threads or 2 of 1024 per SM
        sets = {"hbm": (A.IFR_S_HBM, I.torch_u32_as_i32(1, (4 << 30) // 4, "cuda"), 64),
                "l2": (A.IFR_S_L2, I.torch_u32_as_i32(3, W.L2_SET_BYTES // 4, "cuda"), 256)}
        for name, (kind, buf, rounds) in sets.items():
            for block, bps in ((512, 2), (512, 4), (1024, 2), (256, 4)):
                for staging in (0, 1):
                    if staging and bps * 3 * block * 64 > 200 * 1024:
                        continue  # the ring would not fit beside the other blocks of the SM
                    cfg = ifr.stressor_cfg(kind, sm_count=S, blocks_per_sm=bps, block=block, buf=buf,
                                           working_set_bytes=buf.numel() * 4, staging=staging)
                    P.solo_rate(ctx, cfg, rounds=rounds)
                    rate, res = P.solo_rate(ctx, cfg, rounds=rounds)
                    print(json.dumps({"set": name, "block": block, "blocks_per_sm": bps, "staging": staging,
                                      "status": res["status"], "gbs": round(rate / 1e9, 1)}))
        ctx.close()
        return
    if a.case == "gemm_variants":
        # solo throughput of every GEMM variant at four shapes: the variants take turns
        # (three rounds, so a clock or power drift hits all of them), each turn 3 warm
        # launches and 20 launches timed with CUDA events on the victim stream; best and
        # median of the three
        import statistics

        for M, N, K in ((4096, 4096, 4096), (8192, 8192, 8192), (16384, 12288, 4096), (16384, 4096, 11008)):
            ga = I.torch_normal_bf16(1, M * K, "cuda").view(M, K)
            gb = I.torch_normal_bf16(2, N * K, "cuda").view(N, K)
            gc = torch.empty(M, N, device="cuda")
            res = {v: [] for v in (0, 1, 2, 3, 4)}
            st = {}
            for _round in range(3):
                for var in res:
                    cfg = ifr.victim_cfg(A.IFR_V_GEMM, ga, gb, gc, m=M, n=N, k=K, repeats=3, variant=var)
                    ctx.victim_launch(cfg)
                    cfg.repeats = 20
                    t = ctx.victim_launch(cfg)
                    st[var] = t["status"]
                    res[var].append(2.0 * M * N * K * 20 / (t["event_ms"] * 1e-3) / 1e12)
            for var, r in res.items():
                print(json.dumps({"m": M, "n": N, "k": K, "variant": var, "status": st[var],
                                  "tflops_best": round(max(r), 1), "tflops_median": round(statistics.median(r), 1)}))
            del ga, gb, gc
        ctx.close()
        return
    if a.case == "config5_kernels":
        # one launch of every configuration-5 decoder-layer kernel, in the order of
        # colocate_config5's kernel list (an occupancy capture matches rows by order)
        from paper_2501_16909_b300.colocate_config5 import decoder_kernels

        kern, _t = decoder_kernels(S, "cuda")
        for name, v in kern.items():
            v.repeats = 1
            t = ctx.victim_launch(v)
            print(json.dumps({"kernel": name, "event_ms": round(t["event_ms"], 4), "status": t["status"]}))
        torch.cuda.synchronize()
        ctx.close()
        return
    if a.case == "victim_bandwidth":
        victims, kinds, _t = W.config2_victims("cuda")
        names = {A.IFR_V_GEMV: "gemv", A.IFR_V_LAYERNORM: "layernorm", A.IFR_V_SOFTMAX: "softmax",
                 A.IFR_V_HIST: "hist"}
        for v, k in zip(victims, kinds):
            if k not in names:
                continue
            prof = ctx.victim_profile(v)
            for g in (0, S, 2 * S, 4 * S, 8 * S, 16 * S):
                v.grid, v.repeats = g, 20
                ctx.victim_launch(v)
                t = ctx.victim_launch(v)
                us = t["event_ms"] * 1e3 / 20
                print(json.dumps({"victim": names[k], "grid": g or prof["grid"], "us_per_launch": round(us, 2),
                                  "gbs": round(prof["bytes_per_launch"] / (us * 1e-6) / 1e9, 1)}))
            if k == A.IFR_V_GEMV:
                # the bulk-copy variant (rows streamed into shared memory) on 1 and 2
                # blocks per SM (default: 2)
                v.variant, v.grid = 1, 0
                prof1 = ctx.victim_profile(v)
                for g in (0, S):
                    v.grid, v.repeats = g, 20
                    ctx.victim_launch(v)
                    t = ctx.victim_launch(v)
                    us = t["event_ms"] * 1e3 / 20
                    print(json.dumps({"victim": "gemv variant 1", "grid": g or prof1["grid"],
                                      "us_per_launch": round(us, 2), "status": t["status"],
                                      "gbs": round(prof1["bytes_per_launch"] / (us * 1e-6) / 1e9, 1)}))
                v.variant, v.grid = 0, 0
            # a triad moving the same bytes per launch, timed the same way: the rate a
            # plain stream of this length reaches (launch ramp and tail included)
            n = int(prof["bytes_per_launch"] // 12) // 4 * 4
            tb, tc_ = I.torch_uniform_pm1(90, n, "cuda"), I.torch_uniform_pm1(91, n, "cuda")
            ta = torch.empty(n, device="cuda")
            tv = ifr.victim_cfg(A.IFR_V_TRIAD, tb, tc_, ta, n=n, scalar=0.5, repeats=20)
            ctx.victim_launch(tv)
            t = ctx.victim_launch(tv)
            us = t["event_ms"] * 1e3 / 20
            print(json.dumps({"victim": "triad, same bytes as " + names[k], "n": n, "us_per_launch": round(us, 2),
                              "gbs": round(12.0 * n / (us * 1e-6) / 1e9, 1)}))
            del tb, tc_, ta
        ctx.close()
        return
    if a.case in stressors:
        kind = stressors[a.case]
        bufs = {}
        if kind == A.IFR_S_HBM:
            bufs["hbm"] = I.torch_u32_as_i32(1, (1 << 30) // 4, "cuda")
        if kind == A.IFR_S_L2:
            bufs["l2"] = I.torch_u32_as_i32(3, W.L2_SET_BYTES // 4, "cuda")
        cfg = W.stressor_level_cfg(kind, n_sm, bufs, seed=1)
        if kind in (A.IFR_S_L2, A.IFR_S_HBM):
            cfg.staging = a.staging
        for name, v in (("block", a.block), ("blocks_per_sm", a.bps), ("ilp", a.ilp)):
            if v is not None:
                setattr(cfg, name, v)
        for _ in range(a.repeat):
            rate, res = P.solo_rate(ctx, cfg)
        out.update(rate=rate, unit=P.UNIT[kind] + "/s", elapsed_ms=res["elapsed_ms"], work=res["work"],
                   status=res["status"])
    else:
        victims, kinds, _t = W.config2_victims("cuda")
        names = {A.IFR_V_GEMM: "gemm", A.IFR_V_GEMV: "gemv", A.IFR_V_LAYERNORM: "layernorm",
                 A.IFR_V_SOFTMAX: "softmax", A.IFR_V_HIST: "hist"}
        pick = [v for v, k in zip(victims, kinds) if names[k] == a.case]
        if a.case == "triad":
            wl = W.config1(S)
            pick = wl.victims
        if not pick:
            raise SystemExit("unknown case %r" % a.case)
        v = pick[0]
        v.repeats = 1
        if a.case in ("gemm", "gemv") and a.variant is not None:
            v.variant = a.variant
        for _ in range(a.repeat):
            t = ctx.victim_launch(v)
        out.update(event_ms=t["event_ms"], status=t["status"])
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
