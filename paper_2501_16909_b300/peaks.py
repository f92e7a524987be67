"""Work accounting and peak rates of the stressors' resources.

Each stressor run reports `work` in its kind's unit (chunks, FMA steps per
chain, shared-memory ld/st pairs per lane, tile MMAs, busy blocks); this module
turns that into the algorithmic quantity its resource's peak is stated in, and
provides the peaks:

* HBM        bytes/s — MEASURED_PEAKS.json `hbm_gbs` (STREAM-style copy)
* L2         bytes/s — L2_PEAK_BYTES_PER_S: the rate at which the L2 slices' ports to
                        the crossbar are all busy, from ncu (see the constant)
* FP32 FMA   flop/s  — SMs x 128 lanes x 2 flop x max SM clock
* tensor     flop/s  — SMs x 8192 flop per clock x max SM clock (the pipe's dense rate)
* shared mem wavefronts/s — SMs x 1 wavefront per clock x max SM clock
* scheduler  blocks/s — probe: zero-cycle 32-thread blocks on every SM
* FP64       flop/s  — SMs x 2 fp64 multiplies per clock x max SM clock (B300's
                        1.25 TFLOP/s dense FP64 figure, an FMA counted as two
                        flops; the stressor counts one multiply as one flop)
"""
from __future__ import annotations

import json
import os

from . import _abi as A
from . import stressor_cfg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TILE_MMA_FLOP = 2 * 128 * 128 * 64
UNIT = {A.IFR_S_HBM: "B", A.IFR_S_L2: "B", A.IFR_S_FMA: "flop", A.IFR_S_TENSOR: "flop", A.IFR_S_SMEM_CF: "wavefront",
        A.IFR_S_SMEM_32W: "wavefront", A.IFR_S_SCHED: "block", A.IFR_S_FP64: "flop", A.IFR_S_SLEEP: "round"}
# chunks (block x 64 bytes each) an L2 / HBM stream block reads per round
STREAM_CHUNKS_PER_ROUND = 8
# fixed-work rounds of one calibration run per kind (about a millisecond at full SMs)
CAL_ROUNDS = {A.IFR_S_HBM: 32, A.IFR_S_L2: 128, A.IFR_S_FMA: 32, A.IFR_S_TENSOR: 32, A.IFR_S_SMEM_CF: 16,
              A.IFR_S_SMEM_32W: 32, A.IFR_S_SCHED: 0, A.IFR_S_FP64: 16, A.IFR_S_SLEEP: 10}


# Dense BF16 tcgen05 rate of one SM per clock: 4096 multiply-adds (NVIDIA's 2.25
# PFLOP/s dense BF16 for 148 SMs corresponds to 8192 flop per clock at 1.86 GHz).
TENSOR_FLOP_PER_CLK = 8192
FP64_OPS_PER_CLK = 2  # fp64 multiplies (or FMAs) per clock per SM

# The L2's peak, from ncu on B300 (--clock-control none): for a kernel streaming an
# L2-resident set, lts__t_bytes.sum.per_second / lts__lts2xbar_cycles_active.avg
# .pct_of_peak_sustained_elapsed is the byte rate with the L2-to-crossbar ports 100 %
# busy, the sub-unit that bounds ncu's L2 throughput.  Three different stream kernels
# (17.7 TB/s at 76.2 %, 16.2 TB/s at 69.5 %, 11.4 TB/s at 48.9 % busy) give 23.2
# TB/s within 0.3 %.  A stressor cannot exceed it, unlike a probe of its own best rate.
L2_PEAK_BYTES_PER_S = 23.2e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def ways_of(cfg):
    if cfg.smem_ways:
        return cfg.smem_ways
    return 1 if cfg.kind == A.IFR_S_SMEM_CF else 32


def work_units(cfg, res):
    """Algorithmic work of one stressor run, in UNIT[kind]."""
    k = cfg.kind
    block = cfg.block or {A.IFR_S_L2: 512, A.IFR_S_HBM: 512, A.IFR_S_FMA: 128, A.IFR_S_SMEM_CF: 256,
                          A.IFR_S_SMEM_32W: 256}.get(k, 128)
    w = res["work"]
    if k in (A.IFR_S_HBM, A.IFR_S_L2):
        return w * block * 64
    if k == A.IFR_S_FMA:
        return w * block * (cfg.ilp or 4) * 2
    if k == A.IFR_S_FP64:
        return w * block * (cfg.ilp or 4)
    if k == A.IFR_S_TENSOR:
        return w * TILE_MMA_FLOP
    if k in (A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W):
        return w * (block // 32) * 2 * ways_of(cfg)
    if k in (A.IFR_S_SCHED, A.IFR_S_SLEEP):
        return w
    raise ValueError(k)


def copy_cfg(cfg, **over):
    c = stressor_cfg(cfg.kind)
    for name, _ in cfg._fields_:
        setattr(c, name, getattr(cfg, name))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def solo_rate(ctx, cfg, rounds=None, launches=8):
    """Run a fixed-work copy of cfg alone; returns (rate in UNIT/s, result).

    A duty-cycled run (0 < duty < 1) does four times the rounds: a fixed-work run
    ends inside its last period, so its rate differs from the long-run rate by up to
    (1 - duty) x period over the run's length, which a longer run keeps small."""
    over = {}
    if cfg.kind == A.IFR_S_SCHED:
        over["sched_launches"] = launches
    else:
        over["max_rounds"] = (rounds or CAL_ROUNDS[cfg.kind]) * (4 if 0.0 < cfg.duty < 1.0 else 1)
    res, _ = ctx.run_stressor(copy_cfg(cfg, **over), 30000)
    ms = res["elapsed_ms"]
    return (work_units(cfg, res) / (ms * 1e-3) if ms > 0 else 0.0), res


def peaks(ctx, l2_buf=None):
    """Peak rate per stressor kind (UNIT/s) and where it comes from."""
    m, src = measured_peaks()
    S = ctx.info["num_sms"]
    clk = ctx.info["sm_clock_khz"] * 1e3
    out = {
        A.IFR_S_HBM: (m["hbm_gbs"] * 1e9, "MEASURED_PEAKS hbm_gbs (%s)" % src),
        # the pipe's own rate, not a GEMM's: the stressor's tiles sit in shared memory
        # and it outruns a cuBLAS GEMM (the measured bf16_tflops) by 18 %
        A.IFR_S_TENSOR: (S * TENSOR_FLOP_PER_CLK * clk, "nominal: SMs x 8192 bf16 flop per clock (dense "
                                                        "tcgen05) x max SM clock"),
        A.IFR_S_FMA: (S * 128 * 2 * clk, "nominal: SMs x 128 FP32 lanes x 2 flop x max SM clock"),
        A.IFR_S_SMEM_CF: (S * clk, "nominal: SMs x 1 shared-memory wavefront per clock x max SM clock"),
        A.IFR_S_SMEM_32W: (S * clk, "nominal: SMs x 1 shared-memory wavefront per clock x max SM clock"),
    }
    out[A.IFR_S_L2] = (L2_PEAK_BYTES_PER_S, "ncu: L2-to-crossbar ports fully busy (lts__t_bytes rate over "
                                            "lts__lts2xbar_cycles_active, B300)")
    # B300's dense FP64 figure, 1.25 TFLOP/s with an FMA counted as two flops, is two
    # fp64 operations per clock per SM at the maximum clock; the stressor counts one
    # multiply as one flop, so its peak is two multiplies per clock per SM
    out[A.IFR_S_FP64] = (S * FP64_OPS_PER_CLK * clk, "nominal: SMs x 2 fp64 multiplies per clock (the 1.25 "
                                                      "TFLOP/s dense FP64 figure, FMAs) x max SM clock")
    cfg = stressor_cfg(A.IFR_S_SCHED, sm_count=S, sched_blocks=100000, sched_cycles=1)
    rate, _ = solo_rate(ctx, cfg, launches=8)
    out[A.IFR_S_SCHED] = (rate, "probe: 1-cycle 32-thread blocks on every SM")
    return out
