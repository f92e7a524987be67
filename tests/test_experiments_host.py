"""Host logic of the experiment drivers (no GPU): SM-mask words, medians over pair
runs, and the slowdown table built from sweep cells."""
import pytest

from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import experiments as E
import paper_2501_16909_b300 as ifr


def test_mask_words_and_cfg():
    w = E.mask_bits([0, 31, 32, 147, 255])
    assert w[0] == (1 | 1 << 31) and w[1] == 1 and w[4] == 1 << (147 - 128) and w[7] == 1 << 31
    cfg = E.with_mask(ifr.stressor_cfg(A.IFR_S_FMA), [5, 3, 5, 64])
    assert cfg.mask_mode == 2 and cfg.sm_count == 3
    assert list(cfg.sm_mask)[:3] == [(1 << 3) | (1 << 5), 0, 1]


def _pair(sa, sb, ca, cb, seq, col, ov=1, st=0):
    return dict(solo_a_ns=sa, solo_b_ns=sb, co_a_ns=ca, co_b_ns=cb, seq_ns=seq, col_ns=col, overlapped=ov, status=st)


def test_pair_stats_medians():
    runs = [_pair(100, 100, 200, 150, 200, 200), _pair(110, 90, 220, 180, 200, 250), _pair(90, 95, 900, 100, 185, 900)]
    s = E.pair_stats(runs)
    assert s["slowdown_a"] == pytest.approx(2.0)       # median of 2.0, 2.0, 10.0
    assert s["slowdown_b"] == pytest.approx(1.5)       # median of 1.5, 2.0, 1.0526
    assert s["speedup_seq_over_col"] == pytest.approx(0.8)  # median of 1.0, 0.8, 0.2056
    assert s["all_overlapped"] and s["all_ok"]
    assert not E.pair_stats(runs + [_pair(1, 1, 1, 1, 2, 1, ov=0)])["all_overlapped"]


def _cell(victim, stressor, level, t0, t1, k=1, valid=1):
    c = A.ifr_cell_result()
    c.victim, c.stressor, c.level, c.valid = victim, stressor, level, valid
    c.timing.t_start_ns, c.timing.t_end_ns, c.timing.repeats = t0, t1, k
    return c


def test_slowdowns_from_cells_medians_and_invalid_cells():
    cells = [_cell(0, -1, 0, 0, 100, k=2), _cell(0, -1, 0, 0, 120, k=2), _cell(0, -1, 0, 0, 400, k=2),
             _cell(0, 0, 0, 0, 120, k=2), _cell(0, 0, 1, 0, 240, k=2), _cell(0, 0, 1, 0, 10**6, k=2, valid=0)]
    out = E.slowdowns_from_cells(cells, 1, 2)
    assert out[0]["solo_us"] == pytest.approx(0.06)      # median per-launch time 60 ns
    assert out[0]["slowdown"] == [1.0, 2.0, None]        # invalid cell ignored; level 2 absent
