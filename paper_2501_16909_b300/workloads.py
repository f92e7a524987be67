"""Seeded synthetic workloads for the sweep (inputs live on the GPU).

* config1 — smallest plain case: FP32 triad a = b + 1.5 c, N = 2^22, b and c
  U[-1, 1) from seed 0 (c continues b's stream at index N); HBM stream
  stressor over a 1 GiB int32 buffer (seed 1) at 0 / 25 / 50 / 100 % of the SMs.

Every stressor level is a full ifr_stressor_cfg; level 0 (the stressor launched
on zero SMs) is added by the sweep itself.  Input generation uses ifr_inputs
(SplitMix64), the same recipe the oracle regenerates on the CPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

import ifr_inputs as I

from . import _abi as A
from . import stressor_cfg, victim_cfg

GiB = 1 << 30
MiB = 1 << 20


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


def stream_chunk_bytes(block: int) -> int:
    return block * 64


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
