"""The autotuner on hardware: launch shapes that hit target intensities.

For a real stressor the tuner searches, per target fraction f of the stressor's
all-SM rate, an SM count and, when the SM count alone overshoots, a duty cycle.
Every tuned level must land within +-5 % of its target by the tuner's own
measurement, a fresh measurement of the chosen configuration must agree within
+-10 %, and a target below one SM's share (1/148 of the full rate) can only be
reached with a duty cycle below 1.
"""
import pytest

import ifr_inputs as I
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import autotune
from paper_2501_16909_b300 import peaks as P
from paper_2501_16909_b300 import workloads as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,fractions", [
    (A.IFR_S_FMA, [0.004, 0.125, 0.5, 1.0]),
    (A.IFR_S_HBM, [0.002, 0.25, 0.75]),
])
def test_autotuner_hits_every_target(kind, fractions):
    need_gpu()
    with ifr.Context(0) as ctx:
        S = ctx.info["num_sms"]
        bufs = {"hbm": I.torch_u32_as_i32(1, (1 << 30) // 4, "cuda"), "l2": None}
        base = W.stressor_level_cfg(kind, S, bufs, seed=1)
        tuner = autotune.Tuner(ctx, base, peak=1.0, tol=0.05)
        rmax, levels = tuner.tune(fractions)
        assert rmax > 0
        for lv in levels:
            assert abs(lv.frac_of_max / lv.target - 1.0) <= 0.05, lv
        assert levels[0].sm_count == 1 and levels[0].duty < 1.0, levels[0]
        assert all(lv.duty == 1.0 for lv in levels if lv.target >= 1.0)
        for lv in levels:
            cfg = P.copy_cfg(base, sm_count=lv.sm_count, duty=lv.duty if lv.duty < 1.0 else 0.0)
            r, res = P.solo_rate(ctx, cfg)
            assert res["status"] == 0
            assert abs(r / (lv.target * rmax) - 1.0) <= 0.10, (lv, r / rmax)
