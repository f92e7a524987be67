"""Sweep-plan helpers: per-mode stressor level tables sized from solo victim windows.

A colocated measurement is valid only if the stressor covers the victim's whole
window (Sec. 4.1's constant interference).  Persistent stressors run until they
are stopped, but two quantities must be sized from the victims:

* the scheduler stressor is a finite chain of launches: enough launches to cover
  `margin` x the victim window (one victim in the plain sweep, all victims of the
  batch in the batched sweep);
* every stressor's device deadline: generous multiples of those windows.
"""
from __future__ import annotations

from . import _abi as A
from . import peaks as P


def solo_windows(ctx, victims):
    """First-entry to last-exit span (ns) of each victim's K launches, alone."""
    out = []
    for v in victims:
        t = ctx.victim_launch(v)
        out.append(t["t_end_ns"] - t["t_start_ns"])
    return out


def sched_launch_ns(ctx, levels):
    for row in levels:
        if row and row[0].kind == A.IFR_S_SCHED:
            _, res = P.solo_rate(ctx, row[-1], launches=8)
            return res["elapsed_ms"] * 1e6 / 8
    return 1e5


def mode_levels(levels, windows, t_launch_ns, margin=4.0):
    """(plain, batched) copies of `levels` with launch counts and deadlines set."""
    plain, batched = [], []
    for row in levels:
        prow, brow = [], []
        for cfg in row:
            p = P.copy_cfg(cfg, deadline_ns=int(max(2e9, 40 * max(windows))))
            b = P.copy_cfg(cfg, deadline_ns=int(max(2e9, 40 * sum(windows))))
            if cfg.kind == A.IFR_S_SCHED:
                p.sched_launches = int(min(4096, margin * max(windows) / t_launch_ns + 4))
                b.sched_launches = int(min(65536, margin * sum(windows) / t_launch_ns + 4))
            prow.append(p)
            brow.append(b)
        plain.append(prow)
        batched.append(brow)
    return plain, batched
