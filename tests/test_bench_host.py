"""Host checks of bench.py: the reference arm's JSON line (the oracle timed on the host
cores, no GPU) keeps the bench contract, and the invalid-cell report names the part
of the constant-interference rule (Sec. 4.1) each cell failed."""
import json
import os
import subprocess
import sys
from types import SimpleNamespace as NS

import bench
from paper_2501_16909_b300 import _abi as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    d = json.loads(lines[-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["unit"] == "cells/s" and d["higher_is_better"] is True and d["value"] > 0 and d["ms_per_step"] > 0
    assert "config3" in d["config"]["workload"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]


def _cell(victim=0, stressor=0, level=3, valid=0, t=(100, 200), status=0, s_status=0, active=8,
          s_start_last=90, s_end_first=210, work=0, launched=0):
    return NS(valid=valid, victim=victim, stressor=stressor, level=level,
              timing=NS(status=status, t_start_ns=t[0], t_end_ns=t[1]),
              stress=NS(status=s_status, blocks_active=active, t_start_last_ns=s_start_last,
                        t_end_first_ns=s_end_first, work=work, blocks_launched=launched))


def test_invalid_cells_name_the_failed_rule():
    base = [NS(kind=A.IFR_S_HBM), NS(kind=A.IFR_S_SCHED)]
    vkinds = [A.IFR_V_GEMM, A.IFR_V_SOFTMAX]
    cells = [
        _cell(valid=1),                                             # valid: not listed
        _cell(status=A.IFR_ERR_NOT_RESIDENT),                       # the victim's own status
        _cell(s_status=A.IFR_ERR_TIMEOUT),                          # the stressor's status
        _cell(active=0),                                            # no active stressor block
        _cell(s_start_last=400),                                    # a block started 300 ns after the victim
        _cell(victim=1, stressor=1, s_end_first=199, work=5, launched=9),  # ended 1 ns early (sched)
    ]
    got = bench.invalid_cells(cells, base, vkinds, A)
    assert [g["reason"] for g in got] == [
        "victim status %d" % A.IFR_ERR_NOT_RESIDENT,
        "stressor status %d" % A.IFR_ERR_TIMEOUT,
        "no active stressor block",
        "stressor block started 0.3 us after the victim",
        "stressor block ended 0.0 us before the victim (5 of 9 launched blocks worked)",
    ]
    assert got[0]["victim_kind"] == "gemm" and got[0]["stressor"] == "hbm" and got[0]["level"] == 3
    assert got[-1]["victim_kind"] == "softmax" and got[-1]["stressor"] == "sched"
    assert len(bench.invalid_cells(cells * 4, base, vkinds, A, cap=3)) == 3
