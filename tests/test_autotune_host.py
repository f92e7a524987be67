"""Autotuner host logic against fake solo-rate curves (no GPU): every target fraction
is met within the tolerance when the SM count alone cannot hit it, the duty cycle
repairs overshoots, a target of 1 takes all SMs, and the scheduler stressor (no duty
knob) is tuned by its SM count only."""
import pytest

import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import autotune as T
from paper_2501_16909_b300 import peaks as P

S = 148
FRACTIONS = [(l + 1) / 8 for l in range(8)]


class FakeCtx:
    info = {"num_sms": S}


def _install(monkeypatch, curve):
    """curve(sm_count, duty) -> rate; the duty field is 0 for duty 1."""
    calls = []

    def fake_solo_rate(ctx, cfg, rounds=None, launches=8):
        duty = cfg.duty if cfg.duty > 0 else 1.0
        calls.append((cfg.sm_count, duty))
        return curve(cfg.sm_count, duty), {}

    monkeypatch.setattr(P, "solo_rate", fake_solo_rate)
    return calls


def _tune(kind, tol=0.05):
    t = T.Tuner(FakeCtx(), ifr.stressor_cfg(kind, sm_count=S), peak=1.0, tol=tol)
    return t.tune(FRACTIONS)


def test_linear_curve_hits_every_target_with_sm_count_alone(monkeypatch):
    _install(monkeypatch, lambda n, d: n * d)
    rmax, levels = _tune(A.IFR_S_HBM)
    assert rmax == S
    for lv in levels:
        assert abs(lv.frac_of_max / lv.target - 1) <= 0.05
        assert lv.duty == 1.0
    assert levels[-1].sm_count == S


def test_staircase_undershoot_is_replaced_by_overshoot_and_duty(monkeypatch):
    # rate jumps in steps of 12 SMs: no SM count lands within 5 % of 1/8 of the max
    step = lambda n: 12 * ((n + 11) // 12)
    _install(monkeypatch, lambda n, d: step(n) * d)
    rmax, levels = _tune(A.IFR_S_L2)
    for lv in levels:
        assert abs(lv.frac_of_max / lv.target - 1) <= 0.05, lv
    assert any(lv.duty < 1.0 for lv in levels)


def test_closer_count_below_is_refused_when_outside_tolerance(monkeypatch):
    # a +3 jump at 18 SMs: 17 SMs is the closer count to 1/8 of the max but 10 % short,
    # 18 SMs overshoots by 11 %: the tuner must take 18 and lower the duty
    _install(monkeypatch, lambda n, d: (n if n < 18 else n + 3) * d)
    _rmax, levels = _tune(A.IFR_S_HBM)
    first = levels[0]
    assert first.sm_count == 18 and first.duty < 1.0
    assert abs(first.frac_of_max / first.target - 1) <= 0.05


def test_full_target_takes_all_sms_on_a_non_monotone_top(monkeypatch):
    # the all-SM rate dips below the rate at 139 SMs (two-die L2 behaviour)
    def curve(n, d):
        r = n if n <= 139 else 139 - 0.2 * (n - 139)
        return r * d

    _install(monkeypatch, curve)
    rmax, levels = _tune(A.IFR_S_L2)
    assert levels[-1].sm_count == S
    assert levels[-1].frac_of_max == pytest.approx(1.0)


def test_scheduler_stressor_is_tuned_without_duty(monkeypatch):
    calls = _install(monkeypatch, lambda n, d: 12 * ((n + 11) // 12) * d)
    _rmax, levels = _tune(A.IFR_S_SCHED)
    assert all(lv.duty == 1.0 for lv in levels)
    assert all(d == 1.0 for _n, d in calls)


def test_probes_are_cached(monkeypatch):
    calls = _install(monkeypatch, lambda n, d: n * d)
    _tune(A.IFR_S_FMA)
    assert len(calls) == len(set(calls))


@pytest.mark.parametrize("shape", ["offset", "concave", "noisy_step"])
def test_duty_search_handles_nonproportional_rates(monkeypatch, shape):
    # below one SM's share only the duty cycle can reach the target, and the rate is not
    # proportional to the duty (each on-phase starts with an empty pipeline)
    def duty_part(d):
        if shape == "offset":
            return max(0.0, (d - 0.08) / 0.92)
        if shape == "concave":
            return d ** 0.6
        return max(0.0, d - 0.05) + (0.01 if d > 0.3 else 0.0)

    _install(monkeypatch, lambda n, d: n * (duty_part(d) if d < 1.0 else 1.0))
    t = T.Tuner(FakeCtx(), ifr.stressor_cfg(A.IFR_S_HBM, sm_count=S), peak=1.0, tol=0.05)
    _rmax, levels = t.tune([0.002, 0.004, 0.5])
    for lv in levels:
        assert abs(lv.frac_of_max / lv.target - 1) <= 0.05, (shape, lv)
    assert levels[0].sm_count == 1 and levels[0].duty < 1.0
