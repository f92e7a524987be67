"""Slowdown / sensitivity reduction from raw device timestamps — oracle (test infrastructure).

The paper measures a workload's slowdown as its latency when colocated with a
stressor divided by its latency in isolation (Sec. 4.3, L2 pollution and
bandwidth experiments; Sec. 4.4.1 shared memory), and asks that each stressor
hold a constant interference level for the whole life of the colocated
workload (Sec. 4.1).  It gives no formula for a per-resource sensitivity
vector; the reading used here (one value per stressor kind) is:

  1. per measurement  T = (t_end_max - t_start_min) / K   (K back-to-back launches)
  2. T0 = median of the valid solo repeats; T[r][l] = median over valid repeats
     (even count: mean of the two middle values)
  3. slowdown[r][l] = T[r][l] / T0; level 0 is the stressor launched with zero
     active SMs (the harness runs, nothing interferes)
  4. noise = (max - min) / median of the solo repeats
  5. S[r] = slowdown[r][L] - 1;  AUC[r] = trapezoid of (slowdown - 1) over the
     achieved intensity x (x_0 = 0)
  6. monotone[r]: slowdown[l+1] >= slowdown[l] - 3 * noise for every l
  7. a colocated cell is valid only if the stressor ran without error, had at
     least one active block, every active block had started before the
     victim's first block and none had ended before the victim's last block
  8. symmetric co-run speedup (Table 3): (T_a + T_b) / (max end - min start)

Cells are dicts with keys: victim, stressor (-1 = solo), level, repeat, k,
t_start, t_end, and for colocated cells stress_status, stress_blocks_active,
stress_t_start_last, stress_t_end_first.
"""
from __future__ import annotations

import math


def median(values):
    v = sorted(values)
    n = len(v)
    if n == 0:
        return math.nan
    if n % 2 == 1:
        return float(v[n // 2])
    return (float(v[n // 2 - 1]) + float(v[n // 2])) / 2.0


def duration(cell) -> float:
    return (float(cell["t_end"]) - float(cell["t_start"])) / float(cell["k"])


def cell_valid(cell) -> bool:
    if cell.get("status", 0) != 0:
        return False
    if cell["t_end"] <= cell["t_start"]:
        return False
    if cell["stressor"] < 0:
        return True
    if cell.get("stress_status", 0) != 0:
        return False
    if cell["level"] == 0:
        return True
    if cell.get("stress_blocks_active", 0) <= 0:
        return False
    if cell["stress_t_start_last"] > cell["t_start"]:
        return False
    if cell["stress_t_end_first"] < cell["t_end"]:
        return False
    return True


def sensitivity(cells, victim: int, n_stressors: int, n_levels: int, intensity=None):
    """Reduce one victim's cells.  n_levels counts the stressor levels 1..L;
    level 0 is the zero-SM launch.  intensity[r][l-1] is the achieved fraction
    x_l of level l (default l / L)."""
    mine = [c for c in cells if c["victim"] == victim]
    solo = [duration(c) for c in mine if c["stressor"] < 0 and cell_valid(c)]
    t0 = median(solo)
    noise = (max(solo) - min(solo)) / t0 if solo else math.nan
    L = n_levels
    slow = [[math.nan] * (L + 1) for _ in range(n_stressors)]
    n_valid = len(solo)
    n_invalid = sum(1 for c in mine if c["stressor"] < 0 and not cell_valid(c))
    for r in range(n_stressors):
        for l in range(L + 1):
            ts = []
            for c in mine:
                if c["stressor"] == r and c["level"] == l:
                    if cell_valid(c):
                        ts.append(duration(c))
                        n_valid += 1
                    else:
                        n_invalid += 1
            if ts:
                slow[r][l] = median(ts) / t0
    S, auc, mono = [], [], []
    for r in range(n_stressors):
        xs = [0.0] + [float(intensity[r][l - 1]) if intensity is not None else l / L for l in range(1, L + 1)]
        row = slow[r]
        S.append(row[L] - 1.0)
        if any(math.isnan(v) for v in row):
            auc.append(math.nan)
            mono.append(0)
            continue
        a = 0.0
        for l in range(L):
            a += (xs[l + 1] - xs[l]) * ((row[l] - 1.0) + (row[l + 1] - 1.0)) / 2.0
        auc.append(a)
        ok = all(row[l + 1] >= row[l] - 3.0 * noise for l in range(L))
        mono.append(1 if ok else 0)
    return {
        "t0": t0,
        "noise": noise,
        "slowdown": slow,
        "S": S,
        "auc": auc,
        "monotone": mono,
        "n_valid": n_valid,
        "n_invalid": n_invalid,
    }


def corun_slowdown(solo, corun) -> float:
    """Slowdown of one kernel colocated with another (Sec. 4.3, 4.4.1): its per-launch
    time during the co-run over its per-launch time alone.  Both arguments are
    measurements with keys t_start, t_end, k (rule 1 above)."""
    return duration(corun) / duration(solo)


def corun_speedup(t_a: float, t_b: float, start_a: float, end_a: float, start_b: float, end_b: float) -> float:
    """Sequential over colocated time of two kernels (Table 3's seq/col speedup)."""
    return (t_a + t_b) / (max(end_a, end_b) - min(start_a, start_b))
