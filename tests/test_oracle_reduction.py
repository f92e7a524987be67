"""Pins for the slowdown / sensitivity reduction oracle: forged timestamp logs
whose answers are known by construction."""
import math
import os

import pytest

from oracle import admission
from oracle import reduction as R

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def solo(victim, rep, dur, k=4, t=1000):
    return dict(victim=victim, stressor=-1, level=0, repeat=rep, k=k, t_start=t, t_end=t + dur * k)


def co(victim, r, l, rep, dur, k=4, t=10_000, ok=True):
    return dict(victim=victim, stressor=r, level=l, repeat=rep, k=k, t_start=t, t_end=t + dur * k,
                stress_status=0, stress_blocks_active=8 if l > 0 else 0,
                stress_t_start_last=t - 5 if ok else t + 5, stress_t_end_first=t + dur * k + 5)


def test_median_odd_even():
    assert R.median([3, 1, 2]) == 2
    assert R.median([4, 1, 3, 2]) == 2.5
    assert math.isnan(R.median([]))


def test_forged_2x_log_gives_slowdown_2():
    cells = [solo(0, i, 100) for i in range(3)]
    for l in range(3):
        cells += [co(0, 0, l, i, 100 * (1 + l * 0.5)) for i in range(3)]
    out = R.sensitivity(cells, 0, 1, 2)
    assert out["t0"] == 100
    assert out["noise"] == 0
    assert out["slowdown"][0] == [1.0, 1.5, 2.0]
    assert out["S"] == [1.0]
    # trapezoid over x = 0, 1/2, 1 of (0, 0.5, 1): 0.5 exactly (linear in x)
    assert out["auc"][0] == pytest.approx(0.5, abs=1e-15)
    assert out["monotone"] == [1]


def test_noise_and_monotone_flag():
    cells = [solo(0, 0, 100), solo(0, 1, 110), solo(0, 2, 90)]
    # noise = (110 - 90) / 100 = 0.2; a dip of 0.5 > 3 * 0.2 is not monotone, 0.5 <= 3*0.2 otherwise
    cells += [co(0, 0, 0, 0, 100), co(0, 0, 1, 0, 300), co(0, 0, 2, 0, 250)]
    cells += [co(0, 1, 0, 0, 100), co(0, 1, 1, 0, 300), co(0, 1, 2, 0, 150)]
    out = R.sensitivity(cells, 0, 2, 2)
    assert out["noise"] == pytest.approx(0.2)
    assert out["monotone"] == [1, 0]


def test_invalid_cells_are_dropped():
    cells = [solo(0, 0, 100)]
    cells += [co(0, 0, 0, 0, 100), co(0, 0, 1, 0, 400, ok=False), co(0, 0, 1, 1, 200)]
    out = R.sensitivity(cells, 0, 1, 1)
    assert out["slowdown"][0][1] == 2.0
    assert out["n_invalid"] == 1
    # a stressor that ended before the victim's last block is invalid too
    c = co(0, 0, 1, 2, 200)
    c["stress_t_end_first"] = c["t_end"] - 1
    assert not R.cell_valid(c)
    c = co(0, 0, 1, 2, 200)
    c["stress_status"] = -3
    assert not R.cell_valid(c)


def test_intensity_axis_and_missing_levels():
    cells = [solo(0, 0, 100), co(0, 0, 0, 0, 100), co(0, 0, 1, 0, 200)]
    out = R.sensitivity(cells, 0, 1, 2, intensity=[[0.25, 1.0]])
    assert math.isnan(out["slowdown"][0][2]) and math.isnan(out["auc"][0]) and out["monotone"] == [0]
    cells.append(co(0, 0, 2, 0, 300))
    out = R.sensitivity(cells, 0, 1, 2, intensity=[[0.25, 1.0]])
    # trapezoids: 0.25*(0+1)/2 + 0.75*(1+2)/2
    assert out["auc"][0] == pytest.approx(0.125 + 1.125)


def test_corun_speedup_table3_definition():
    # two kernels of 10 ms each that overlap perfectly in 10.36 ms give 1.93x
    assert R.corun_speedup(10, 10, 0, 10.36, 0, 10.36) == pytest.approx(20 / 10.36)
    # fully serialised co-run gives 1
    assert R.corun_speedup(10, 10, 0, 10, 10, 20) == 1.0


def test_register_admission_paper_example():
    kv = {}
    with open(os.path.join(GOLD, "register_admission_h100.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                kv[a] = int(b)
    used = kv["stressor_regs_per_thread"] * kv["stressor_threads_per_block"]
    assert admission.free_after(kv["regs_per_sm"], used, 1) == kv["expected_free_regs"]
    sm = dict(blocks=32, threads=2048, regs=kv["regs_per_sm"], smem=228 * 1024)
    stress = dict(threads=128, regs=used, smem=0)
    victim = dict(threads=1024, regs=kv["victim_regs_per_block"], smem=0)
    assert admission.admits(sm, [stress], victim) == bool(kv["expected_admitted"])
    assert admission.admits(sm, [], victim)


def test_corun_slowdown_forged_logs():
    # a victim whose 3 launches take 2x as long beside the co-runner, counted per launch
    alone = dict(t_start=100, t_end=100 + 3 * 500, k=3)
    both = dict(t_start=9000, t_end=9000 + 3 * 1000, k=3)
    assert R.corun_slowdown(alone, both) == 2.0
    # different launch counts on the two sides: per-launch times, not spans
    chain_alone = dict(t_start=0, t_end=700, k=1)
    chain_co = dict(t_start=0, t_end=10 * 770, k=10)
    assert math.isclose(R.corun_slowdown(chain_alone, chain_co), 1.1, rel_tol=1e-12)
