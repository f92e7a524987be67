"""Autotuner: launch shapes that hit target stressor intensities.

For one stressor kind and a list of target fractions f (of the stressor's own
full-intensity rate, i.e. all SMs at duty 1), find for each f a configuration
(sm_count, duty) whose solo fixed-work rate is within +-5 % of f * rate_max:

  1. bisect on sm_count (the rate grows monotonically with the SMs used) for the
     smallest count whose rate reaches the target; the count just below replaces it
     when that one is closer and within the tolerance; a target of 1 takes all SMs;
  2. if that overshoots by more than the tolerance, lower the duty cycle
     (active fraction of each period): start at the measured ratio, then keep a
     bracket around the target and refine by regula falsi (bisecting when the
     secant leaves the bracket), up to eight probes.

Every probe is one solo run through the C ABI (ifr_stressor_launch with
max_rounds, CUDA events on the stressor stream); results are cached per
(sm_count, duty).  The scheduler stressor has no duty cycle: it is tuned by
sm_count only.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import _abi as A
from . import peaks as P


@dataclass
class Level:
    target: float        # target fraction of rate_max
    sm_count: int
    duty: float
    rate: float          # achieved rate (UNIT/s)
    frac_of_max: float   # rate / rate_max
    frac_of_peak: float  # rate / resource peak
    probes: int


class Tuner:
    def __init__(self, ctx, base_cfg, peak: float, tol: float = 0.05, rounds=None):
        self.ctx = ctx
        self.base = base_cfg
        self.peak = peak
        self.tol = tol
        self.rounds = rounds
        self.cache = {}
        self.S = ctx.info["num_sms"]
        self.probes = 0

    def rate(self, sm_count: int, duty: float = 1.0) -> float:
        key = (sm_count, round(duty, 4))
        if key not in self.cache:
            cfg = P.copy_cfg(self.base, sm_count=sm_count, duty=float(duty) if duty < 1.0 else 0.0)
            if self.base.kind == A.IFR_S_SCHED:
                r, _ = P.solo_rate(self.ctx, cfg, launches=8)
            else:
                r, _ = P.solo_rate(self.ctx, cfg, rounds=self.rounds)
            self.cache[key] = r
            self.probes += 1
        return self.cache[key]

    def tune_duty(self, n: int, target: float, r_full: float, max_probes: int = 8):
        """Duty cycle at n SMs whose rate is within the tolerance of `target`.  The rate
        rises with the duty (0 at duty 0, r_full at 1) but not in proportion: every
        on-phase starts with an empty pipeline, so short on-phases deliver less.  The
        search keeps a bracket [lo, hi] around the target and takes the secant
        (regula falsi) inside it, bisecting when the secant leaves the bracket; it
        returns the closest probe."""
        lo_d, lo_r, hi_d, hi_r = 0.0, 0.0, 1.0, r_full
        best = (abs(r_full / target - 1), 1.0, r_full)
        d = max(0.02, min(1.0, target / r_full))
        for _ in range(max_probes):
            rd = self.rate(n, d)
            err = abs(rd / target - 1)
            if err < best[0]:
                best = (err, d, rd)
            if err <= self.tol:
                break
            if rd > target:
                hi_d, hi_r = d, rd
            else:
                lo_d, lo_r = d, rd
            nd = lo_d + (target - lo_r) * (hi_d - lo_d) / (hi_r - lo_r) if hi_r > lo_r else 0.5 * (lo_d + hi_d)
            if not lo_d < nd < hi_d:
                nd = 0.5 * (lo_d + hi_d)
            d = max(0.02, nd)
        return best[1], best[2]

    def tune(self, fractions):
        rmax = self.rate(self.S)
        out = []
        for f in fractions:
            target = f * rmax
            p0 = self.probes
            lo, hi = 1, self.S
            if self.rate(lo) >= target:
                hi = lo
            while lo < hi:
                mid = (lo + hi) // 2
                if self.rate(mid) >= target:
                    hi = mid
                else:
                    lo = mid + 1
            n = self.S if f >= 1.0 else hi  # the full rate is the all-SM rate by definition
            # the count just below may land closer to the target than the first one above
            # it; take it only when it is within the tolerance (an undershoot cannot be
            # repaired with the duty cycle, an overshoot can)
            if (n == hi and n > 1 and abs(self.rate(n - 1) - target) < abs(self.rate(n) - target)
                    and abs(self.rate(n - 1) / target - 1) <= self.tol):
                n -= 1
            duty, r = 1.0, self.rate(n)
            if self.base.kind != A.IFR_S_SCHED and r > target * (1 + self.tol):
                duty, r = self.tune_duty(n, target, r)
            out.append(Level(f, n, duty, r, r / rmax, r / self.peak if self.peak else float("nan"),
                             self.probes - p0))
        return rmax, out


def tuned_levels(ctx, base_cfgs, peaks, fractions, tol=0.05):
    """Tune every stressor of `base_cfgs` (one full-intensity cfg per kind).
    Returns (levels[n_stressors][n_levels] of ifr_stressor_cfg, report)."""
    levels, report = [], []
    for cfg in base_cfgs:
        t = Tuner(ctx, cfg, peaks[cfg.kind][0], tol)
        rmax, lv = t.tune(fractions)
        row = [P.copy_cfg(cfg, sm_count=l.sm_count, duty=(l.duty if l.duty < 1.0 else 0.0)) for l in lv]
        levels.append(row)
        report.append({"kind": A.STRESSOR_NAMES[cfg.kind], "rate_max": rmax, "probes": t.probes,
                       "levels": [l.__dict__ for l in lv]})
    return levels, report
