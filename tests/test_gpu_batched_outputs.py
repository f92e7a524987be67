"""Victim outputs written inside the graph-captured batched sweep.

The batched sweep replays, per (stressor, level), one CUDA graph in which all
victims run back to back beside a running stressor.  This is the one path where
colocation could corrupt results (a stressor and a victim sharing TMEM, shared
memory and the L2), so after a batched sweep every victim's output is compared
with the oracle: ten configuration-3 victims of uneven shapes (four GEMMs, one of
676 output tiles on 148 SMs, so the last wave is ragged; two GEMVs, two softmax,
two layernorm) beside a full HBM stream stressor and a full tensor-pipe stressor.
Outputs are filled with NaN first, so an output the sweep never wrote fails.  The
same check runs on the grouped batched sweep, where victims of one row kernel share
one persistent launch.
"""
import numpy as np
import pytest
import torch

import ifr_inputs as I
import oracle
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import workloads as W
from tests.gpu_common import BF16_TOL, assert_fp32_close, need_gpu

pytestmark = pytest.mark.gpu

SUBSET = [0, 1, 6, 8, 19, 22, 33, 37, 50, 60]


def _bf16_bits(seed, n):
    return oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(seed, np.arange(n)))


def _bf16_values(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _check_gemm(i, shape, C_gpu, rng):
    _, M, N, K = shape
    s = W.config3_seeds(i)
    Ab = _bf16_bits(s, M * K).reshape(M, K)
    Bb = _bf16_bits(s + 1, N * K).reshape(N, K)
    got = C_gpu.double().cpu().numpy()
    assert np.isfinite(got).all()
    # a few entries of every 128 x 128 output block against the oracle's fp64 dot products
    ij = []
    for bm in range(M // 128):
        for bn in range(N // 128):
            for _ in range(3):
                ij.append((bm * 128 + rng.integers(0, 128), bn * 128 + rng.integers(0, 128)))
    ij = np.array(ij, np.int64)
    ref = oracle.gemm_entries(Ab, Bb, ij)
    g = got[ij[:, 0], ij[:, 1]]
    rms = np.sqrt(np.mean(ref * ref))
    assert np.all(np.abs(g - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms)), i
    if M * N * K <= 1 << 32:
        # small GEMMs: every entry against the fp64 product of the same bf16 values
        full = _bf16_values(Ab) @ _bf16_values(Bb).T
        rms = np.sqrt(np.mean(full * full))
        assert np.all(np.abs(got - full) <= BF16_TOL * np.maximum(np.abs(full), rms)), i
        assert np.linalg.norm(got - full) <= BF16_TOL * np.linalg.norm(full), i


# grouped: the two GEMVs, the two softmax and the two layernorm victims each run as one
# grouped persistent launch that walks both victims' rows, and the GEMMs as two grouped
# launches (one per tile width, one of them 682 tiles of two problems)
@pytest.mark.parametrize("grouped", [False, True])
def test_batched_sweep_victim_outputs_match_oracle(grouped):
    need_gpu()
    shapes = W.config3_shapes()
    with ifr.Context(0) as ctx:
        S = ctx.info["num_sms"]
        victims, kinds, t = W.config3_victims("cuda", only=SUBSET)
        assert len(victims) == len(SUBSET)
        assert shapes[1][0] == "gemm" and (shapes[1][1] // 128) * (shapes[1][2] // 256) % S != 0
        for i in SUBSET:
            t[i][-1].fill_(float("nan"))
        bufs = {"hbm": I.torch_u32_as_i32(1, (1 << 30) // 4, "cuda"), "l2": None}
        levels = [[W.stressor_level_cfg(A.IFR_S_HBM, S, bufs, seed=1)],
                  [W.stressor_level_cfg(A.IFR_S_TENSOR, S, bufs, seed=2)]]
        if grouped:
            # the same sweep ungrouped first, for its launch count
            n0 = ctx.launch_count()
            ctx.sweep(victims, levels, repeats=1, batched=True)
            ungrouped = ctx.launch_count() - n0
            for i in SUBSET:
                t[i][-1].fill_(float("nan"))
        n0 = ctx.launch_count()
        cells = ctx.sweep(victims, levels, repeats=1, batched=True, grouped=grouped)
        launches = ctx.launch_count() - n0
        assert len(cells) == len(victims) * (1 + 2 * 2)
        # every victim measured on its own record, also inside a grouped launch
        assert all(c.timing.t_end_ns > c.timing.t_start_ns > 0 and c.timing.blocks > 0 for c in cells)
        co = [c for c in cells if c.stressor >= 0 and c.level == 1]
        assert all(c.stress.blocks_active == c.stress.planned_active > 0 for c in co)
        assert sum(c.valid for c in co) >= 0.8 * len(co)
        torch.cuda.synchronize()
    if grouped:
        # 5 graphs (solo, two levels of two stressors), each with 5 grouped launches in
        # place of 10 single-victim launches (two GEMMs of each tile width, two GEMVs,
        # two softmax, two layernorm)
        assert launches == ungrouped - 5 * 5
    rng = np.random.default_rng(0)
    for i in SUBSET:
        kind, a, b, c = shapes[i]
        s = W.config3_seeds(i)
        out = t[i][-1]
        if kind == "gemm":
            _check_gemm(i, shapes[i], out, rng)
        elif kind == "gemv":
            R, Wd = a, c
            Ab = _bf16_bits(s, R * Wd).reshape(R, Wd)
            xb = _bf16_bits(s + 1, Wd)
            ref = oracle.gemv_rows(Ab, xb, np.arange(R))
            got = out.double().cpu().numpy()
            rms = np.sqrt(np.mean(ref * ref))
            assert np.all(np.abs(got - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms)), i
        else:
            R, Wd = a, b
            xs = I.np_uniform_pm1(s, np.arange(R * Wd)).reshape(R, Wd)
            ref = (oracle.softmax_rows(xs, np.arange(R)) if kind == "softmax"
                   else oracle.layernorm_rows(xs, np.arange(R), 1e-5))
            assert_fp32_close(out.cpu().numpy(), ref)
