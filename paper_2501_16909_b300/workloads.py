"""Seeded synthetic workloads for the sweep (inputs live on the GPU).

* config1 — smallest plain case: FP32 triad a = b + 1.5 c, N = 2^22, b and c
  U[-1, 1) from seed 0 (c continues b's stream at index N); HBM stream
  stressor over a 1 GiB int32 buffer (seed 1) at 0 / 25 / 50 / 100 % of the SMs.

Every stressor level is a full ifr_stressor_cfg; level 0 (the stressor launched
on zero SMs) is added by the sweep itself.  Input generation uses ifr_inputs
(SplitMix64), the same recipe the oracle regenerates on the CPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

import ifr_inputs as I

from . import _abi as A
from . import stressor_cfg, victim_cfg

GiB = 1 << 30
MiB = 1 << 20
# L2-resident stressor set, sized from the measured L2: with every SM streaming, a
# B300 sustains 14-16 TB/s from L2 up to a 16 MiB set and falls to 6.5-12 TB/s at
# 48 MiB, so the L2 stressor streams 16 MiB (the configuration's "48 MB" was
# written against a 50 MB H100 L2).
L2_SET_BYTES = 16 * MiB


@dataclass
class Workload:
    name: str
    victims: list
    levels: list                     # [n_stressors][n_levels] ifr_stressor_cfg
    fractions: list                  # SM fraction of each level (1..L)
    stressor_kinds: list
    victim_kinds: list
    tensors: dict = field(default_factory=dict)
    repeats: int = 3
    h2d_bytes: int = 0               # bytes of inputs a host-resident run copies in
    d2h_bytes: int = 0               # bytes of outputs it copies back

    @property
    def n_cells(self):
        ns = len(self.levels)
        nl = len(self.levels[0]) if ns else 0
        return self.repeats * len(self.victims) * (1 + ns * (nl + 1))


def config1(num_sms: int, device="cuda", hbm_bytes: int = GiB, n: int = 1 << 22, repeats: int = 3,
            launches_per_measurement: int = 8) -> Workload:
    b = I.torch_uniform_pm1(0, n, device)
    c = I.torch_uniform_pm1(0, n, device, start=n)
    a = torch.empty(n, device=device)
    buf = I.torch_u32_as_i32(1, hbm_bytes // 4, device)
    victims = [victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=1.5, repeats=launches_per_measurement)]
    fr = [0.25, 0.5, 1.0]
    lv = [[stressor_cfg(A.IFR_S_HBM, sm_count=max(1, round(f * num_sms)), blocks_per_sm=2, block=512,
                        working_set_bytes=hbm_bytes, buf=buf, seed=1) for f in fr]]
    return Workload("config1: triad N=2^22 x HBM stream 1 GiB at 0/25/50/100% SMs", victims, lv, fr,
                    [A.IFR_S_HBM], [A.IFR_V_TRIAD], dict(a=a, b=b, c=c, buf=buf), repeats,
                    h2d_bytes=b.numel() * 4 + c.numel() * 4 + buf.numel() * 4, d2h_bytes=a.numel() * 4)


# ----------------------------------------------------------------------------- config 2
# Stressor footprints per SM (threads / blocks): kept small so that victim blocks
# can be co-resident (the paper's stressors use one 128-thread block per SM).
STRESSOR_DEFAULTS = {
    A.IFR_S_SCHED: dict(sched_blocks=100000, sched_cycles=100),
    A.IFR_S_FMA: dict(block=128, blocks_per_sm=2, ilp=8),
    A.IFR_S_TENSOR: dict(blocks_per_sm=1),
    A.IFR_S_SMEM_CF: dict(block=256, blocks_per_sm=2),
    A.IFR_S_SMEM_32W: dict(block=256, blocks_per_sm=2),
    # two blocks of 512 hold the same threads and registers per SM as four of 256;
    # with the word-load stream kernel they keep the L2-to-crossbar ports 76.3 % busy
    # against 73.0 %, at the same ALU share (9.4 % against 9.3 %; ncu, B300, same box).
    # One block of 1024 reached 78.6 % but runs the kernel with its block size read at
    # run time, whose per-chunk fold takes the ALU to 12.4 %.
    A.IFR_S_L2: dict(block=512, blocks_per_sm=2),
    A.IFR_S_HBM: dict(block=512, blocks_per_sm=2),
    # two blocks of 256, 8 chains each: the fp64 pipe 84.0 % active (ncu) against 80.0 %
    # for the paper's one 128-thread block per SM with 4 chains (Sec. 4.4.3), which the
    # Table 3 experiment keeps
    A.IFR_S_FP64: dict(block=256, blocks_per_sm=2, ilp=8),
}

VICTIM_LAUNCHES = {A.IFR_V_GEMM: 4, A.IFR_V_GEMV: 16, A.IFR_V_LAYERNORM: 4, A.IFR_V_SOFTMAX: 4, A.IFR_V_HIST: 8,
                   A.IFR_V_TRIAD: 8}


def config2_victims(device="cuda"):
    """BF16 GEMM 4096^3 (N(0,1)), BF16 GEMV 8192^2, FP32 layernorm 16384x4096,
    FP32 row softmax 8192^2, int32 histogram of 2^26 keys (seeds 11..16)."""
    t = {}
    G = 4096
    t["gA"] = I.torch_normal_bf16(11, G * G, device).view(G, G)
    t["gB"] = I.torch_normal_bf16(12, G * G, device).view(G, G)
    t["gC"] = torch.empty(G, G, device=device)
    R = 8192
    t["vA"] = I.torch_normal_bf16(13, R * R, device).view(R, R)
    t["vx"] = I.torch_normal_bf16(14, R, device)
    t["vy"] = torch.empty(R, device=device)
    t["lx"] = I.torch_uniform_pm1(15, 16384 * 4096, device).view(16384, 4096)
    t["ly"] = torch.empty_like(t["lx"])
    t["sx"] = I.torch_uniform_pm1(16, R * R, device).view(R, R)
    t["sy"] = torch.empty_like(t["sx"])
    t["hk"] = I.torch_key256(2, 1 << 26, device)
    t["hb"] = torch.zeros(256, dtype=torch.int32, device=device)
    L = VICTIM_LAUNCHES
    victims = [
        victim_cfg(A.IFR_V_GEMM, t["gA"], t["gB"], t["gC"], m=G, n=G, k=G, repeats=L[A.IFR_V_GEMM]),
        victim_cfg(A.IFR_V_GEMV, t["vA"], t["vx"], t["vy"], m=R, k=R, repeats=L[A.IFR_V_GEMV]),
        victim_cfg(A.IFR_V_LAYERNORM, t["lx"], None, t["ly"], m=16384, n=4096, repeats=L[A.IFR_V_LAYERNORM]),
        victim_cfg(A.IFR_V_SOFTMAX, t["sx"], None, t["sy"], m=R, n=R, repeats=L[A.IFR_V_SOFTMAX]),
        victim_cfg(A.IFR_V_HIST, t["hk"], None, t["hb"], n=1 << 26, repeats=L[A.IFR_V_HIST]),
    ]
    kinds = [A.IFR_V_GEMM, A.IFR_V_GEMV, A.IFR_V_LAYERNORM, A.IFR_V_SOFTMAX, A.IFR_V_HIST]
    return victims, kinds, t


def stressor_level_cfg(kind, sm_count, bufs, seed=0, **over):
    kw = dict(STRESSOR_DEFAULTS[kind])
    kw.update(over)
    if kind == A.IFR_S_L2:
        kw.update(buf=bufs["l2"], working_set_bytes=bufs["l2"].numel() * 4)
    elif kind == A.IFR_S_HBM:
        kw.update(buf=bufs["hbm"], working_set_bytes=bufs["hbm"].numel() * 4)
    return stressor_cfg(kind, sm_count=sm_count, seed=seed, **kw)


def config2(num_sms: int, device="cuda", n_levels: int = 8, repeats: int = 3, hbm_bytes: int = 4 * GiB,
            l2_bytes: int = L2_SET_BYTES) -> Workload:
    victims, vkinds, t = config2_victims(device)
    t["l2"] = I.torch_u32_as_i32(3, l2_bytes // 4, device)
    t["hbm"] = I.torch_u32_as_i32(1, hbm_bytes // 4, device)
    kinds = [A.IFR_S_SCHED, A.IFR_S_FMA, A.IFR_S_TENSOR, A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W, A.IFR_S_L2, A.IFR_S_HBM]
    fr = [(l + 1) / n_levels for l in range(n_levels)]
    levels = [[stressor_level_cfg(k, max(1, round(f * num_sms)), t, seed=r + 1) for f in fr]
              for r, k in enumerate(kinds)]
    h2d = sum(v.numel() * v.element_size() for k, v in t.items() if k in ("gA", "gB", "vA", "vx", "lx", "sx", "hk",
                                                                          "l2", "hbm"))
    d2h = sum(t[k].numel() * t[k].element_size() for k in ("gC", "vy", "ly", "sy", "hb"))
    return Workload("config2: 7 stressors x 8 SM-fraction levels x 5 victims (GEMM 4096^3, GEMV 8192^2, "
                    "LN 16384x4096, softmax 8192^2, histogram 2^26)", victims, levels, fr, kinds, vkinds, t,
                    repeats, h2d_bytes=h2d, d2h_bytes=d2h)


# ----------------------------------------------------------------------------- config 3
def _loguniform(u64: int, lo: int, hi: int, mult: int) -> int:
    """Log-uniform draw in [lo, hi] from one generator output, rounded to a multiple of mult."""
    u01 = (int(u64) >> 11) * 2.0 ** -53
    v = math.exp(math.log(lo) + u01 * (math.log(hi) - math.log(lo)))
    r = mult * int(round(v / mult))
    return int(min(hi - hi % mult, max(lo, r)))


def config3_shapes(seed: int = 3):
    """64 uneven victims: 16 GEMMs (M, N, K log-uniform in [256, 8192], multiples of
    128), 16 GEMVs (rows log-uniform in [1024, 16384], width 4096), 16 softmax and 16
    layernorm (rows log-uniform in [512, 32768], width 4096).  Draw i of the seed's
    SplitMix64 stream feeds the i-th dimension in that order."""
    u = I.np_u64(seed, np.arange(96))
    shapes = []
    for g in range(16):
        M, N, K = (_loguniform(u[3 * g + j], 256, 8192, 128) for j in range(3))
        shapes.append(("gemm", M, N, K))
    for g in range(16):
        shapes.append(("gemv", _loguniform(u[48 + g], 1024, 16384, 1), 0, 4096))
    for g in range(16):
        shapes.append(("softmax", _loguniform(u[64 + g], 512, 32768, 1), 4096, 0))
    for g in range(16):
        shapes.append(("layernorm", _loguniform(u[80 + g], 512, 32768, 1), 4096, 0))
    return shapes


def config3_seeds(i: int) -> int:
    """Input seed of config-3 victim i (its second input uses the next seed)."""
    return 100 + 4 * i


def config3_victims(device="cuda", seed: int = 3, launches: int = 1, only=None):
    """Allocate and fill the 64 config-3 victims (inputs seeded per victim index),
    or only the victims whose indices are listed in `only` (same shapes and seeds)."""
    t, victims, kinds = {}, [], []
    for i, (kind, a, b, c) in enumerate(config3_shapes(seed)):
        if only is not None and i not in only:
            continue
        s = config3_seeds(i)
        if kind == "gemm":
            M, N, K = a, b, c
            A_ = I.torch_normal_bf16(s, M * K, device).view(M, K)
            B_ = I.torch_normal_bf16(s + 1, N * K, device).view(N, K)
            C_ = torch.empty(M, N, device=device)
            t[i] = (A_, B_, C_)
            victims.append(victim_cfg(A.IFR_V_GEMM, A_, B_, C_, m=M, n=N, k=K, repeats=launches))
            kinds.append(A.IFR_V_GEMM)
        elif kind == "gemv":
            R, W = a, c
            A_ = I.torch_normal_bf16(s, R * W, device).view(R, W)
            x = I.torch_normal_bf16(s + 1, W, device)
            y = torch.empty(R, device=device)
            t[i] = (A_, x, y)
            victims.append(victim_cfg(A.IFR_V_GEMV, A_, x, y, m=R, k=W, repeats=launches))
            kinds.append(A.IFR_V_GEMV)
        else:
            R, W = a, b
            x = I.torch_uniform_pm1(s, R * W, device).view(R, W)
            y = torch.empty_like(x)
            t[i] = (x, y)
            k = A.IFR_V_SOFTMAX if kind == "softmax" else A.IFR_V_LAYERNORM
            victims.append(victim_cfg(k, x, None, y, m=R, n=W, repeats=launches))
            kinds.append(k)
    return victims, kinds, t


def config3_base_stressors(num_sms: int, bufs, kinds=None):
    """Full-intensity configuration of every stressor kind (the autotuner's start)."""
    kinds = kinds or [A.IFR_S_SCHED, A.IFR_S_FMA, A.IFR_S_TENSOR, A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W, A.IFR_S_L2,
                      A.IFR_S_HBM]
    return [stressor_level_cfg(k, num_sms, bufs, seed=r + 1) for r, k in enumerate(kinds)]


# ----------------------------------------------------------------------------- probes
def probe_victims(num_sms, device="cuda"):
    """Six small kernels whose slowdown beside a co-runner measures the co-runner's
    pressure on one resource each (the predictor's co-runner features), in the order
    of predictor.PROBES: an HBM-bound triad (2^24 elements, 192 MiB), an L2-resident
    triad (2^19 elements, 6 MiB), a tensor-pipe GEMM (2048 x 2048 x 1024), a
    shared-memory-atomic histogram (2^22 keys), an exp-bound softmax (4096 x 1024) and
    a GEMV of 65536 short rows (64 columns: many light blocks).  Seeds 300..315."""
    t = {}
    n = 1 << 24
    t["hb"], t["hc"], t["ha"] = (I.torch_uniform_pm1(300, n, device), I.torch_uniform_pm1(301, n, device),
                                 torch.empty(n, device=device))
    m = 1 << 19
    t["lb"], t["lc"], t["la"] = (I.torch_uniform_pm1(302, m, device), I.torch_uniform_pm1(303, m, device),
                                 torch.empty(m, device=device))
    t["gA"] = I.torch_normal_bf16(304, 2048 * 1024, device).view(2048, 1024)
    t["gB"] = I.torch_normal_bf16(305, 2048 * 1024, device).view(2048, 1024)
    t["gC"] = torch.empty(2048, 2048, device=device)
    t["hk"] = I.torch_key256(306, 1 << 22, device)
    t["hbins"] = torch.zeros(256, dtype=torch.int32, device=device)
    t["sx"] = I.torch_uniform_pm1(307, 4096 * 1024, device).view(4096, 1024)
    t["sy"] = torch.empty_like(t["sx"])
    t["vA"] = I.torch_normal_bf16(308, 65536 * 64, device).view(65536, 64)
    t["vx"] = I.torch_normal_bf16(309, 64, device)
    t["vy"] = torch.empty(65536, device=device)
    probes = [
        victim_cfg(A.IFR_V_TRIAD, t["hb"], t["hc"], t["ha"], n=n, scalar=1.5),
        victim_cfg(A.IFR_V_TRIAD, t["lb"], t["lc"], t["la"], n=m, scalar=1.5),
        victim_cfg(A.IFR_V_GEMM, t["gA"], t["gB"], t["gC"], m=2048, n=2048, k=1024),
        victim_cfg(A.IFR_V_HIST, t["hk"], None, t["hbins"], n=1 << 22),
        victim_cfg(A.IFR_V_SOFTMAX, t["sx"], None, t["sy"], m=4096, n=1024),
        victim_cfg(A.IFR_V_GEMV, t["vA"], t["vx"], t["vy"], m=65536, k=64),
    ]
    return probes, t
