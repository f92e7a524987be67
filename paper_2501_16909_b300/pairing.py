"""Colocation rules of two schedulers the paper critiques, set against the slowdown
predictor on measured kernel pairs (Sec. 3, Pitfalls 1 and 2; Sec. 5 asks for an
estimator that sees every resource instead).

* Usher's rule (Pitfall 1, Sec. 2 "achieved occupancy"): two kernels may share the
  GPU when their achieved occupancies, each taken from a solo profile (ncu
  ``sm__warps_active.avg.pct_of_peak_sustained_active``), add up to less than 100 %.
* Orion's rule (Pitfall 2, Sec. 2 "arithmetic intensity"): a kernel is compute-bound
  when its arithmetic intensity (flops per DRAM byte) reaches the ridge point of the
  pipe it computes on (that pipe's peak flop/s over the peak HBM byte/s), otherwise
  memory-bound; two kernels may share the GPU when one is compute-bound and the other
  memory-bound.
* The predictor's rule: share when the predicted slowdown of the victim stays within
  the slowdown bound the colocation has to keep.
* The per-resource estimator's rule: the same with 1 + max_r S_v,r(x_c,r).

A measured pair is directional (victim beside co-runner, the victim's slowdown).  A
rule that decides per unordered pair gives the same answer to both directions.  Each
rule is scored at several bounds: the pairs it colocates, its violations (colocated,
measured slowdown above the bound), the pairs it misses (refused, measured within the
bound), precision and recall.  Pure host code.

    python -m paper_2501_16909_b300.pairing <config-5 JSON> <ncu occupancy CSV>

re-scores a saved configuration-5 result (``colocate_config5`` output with
``kernel_info``) against an occupancy capture of its kernels.
"""
from __future__ import annotations

import csv
import io
import json
import sys

OCCUPANCY_METRIC = "sm__warps_active.avg.pct_of_peak_sustained_active"
BOUNDS = (1.1, 1.25, 1.5, 2.0)


def parse_ncu_occupancy(text: str) -> list:
    """[(kernel name, achieved occupancy as a fraction)] in launch order from the CSV
    that ``ncu --metrics sm__warps_active.avg.pct_of_peak_sustained_active --csv``
    writes (its ``==PROF==`` / ``==WARNING==`` lines are skipped)."""
    rows = [ln for ln in text.splitlines() if ln.startswith('"')]
    out = []
    for r in csv.DictReader(io.StringIO("\n".join(rows))):
        if r.get("Metric Name") != OCCUPANCY_METRIC:
            continue
        out.append((int(r["ID"]), r["Kernel Name"], float(r["Metric Value"].replace(",", "")) / 100.0))
    out.sort()
    return [(name, v) for _id, name, v in out]


def usher_colocate(occ_a: float, occ_b: float) -> bool:
    """Sum of achieved occupancies below 100 % (occupancies as fractions)."""
    return occ_a + occ_b < 1.0


def orion_class(flops: float, nbytes: float, uses_tensor: bool, peaks: dict) -> str:
    """'compute' when flops / bytes reaches the ridge point of the kernel's pipe."""
    pipe = peaks["tensor"] if uses_tensor else peaks["fp32"]
    ridge = pipe / peaks["hbm"]
    ai = flops / nbytes if nbytes > 0 else float("inf")
    return "compute" if ai >= ridge else "memory"


def orion_colocate(cls_a: str, cls_b: str) -> bool:
    """Complementary profiles: one compute-bound, one memory-bound."""
    return cls_a != cls_b


def score(colocate, measured, bound: float) -> dict:
    """Decisions against measured victim slowdowns at one bound."""
    assert len(colocate) == len(measured)
    ok = [m <= bound for m in measured]
    n_col = sum(1 for c in colocate if c)
    good_col = sum(1 for c, g in zip(colocate, ok) if c and g)
    viol = n_col - good_col
    missed = sum(1 for c, g in zip(colocate, ok) if g and not c)
    n_ok = sum(ok)
    worst = max((m for c, m in zip(colocate, measured) if c), default=None)
    return {
        "bound": bound, "pairs": len(measured), "within_bound": n_ok, "colocated": n_col, "violations": viol,
        "missed": missed, "precision": round(good_col / n_col, 4) if n_col else None,
        "recall": round(good_col / n_ok, 4) if n_ok else None,
        "worst_colocated": round(worst, 4) if worst is not None else None,
    }


def decisions(pairs, kernel_info, occupancy, peaks, bound):
    """{rule: [colocate?] per pair} at one bound (only the predictor rules use it)."""
    cls = {n: orion_class(k["flops"], k["bytes"], k["uses_tensor"], peaks) for n, k in kernel_info.items()}
    return {
        "usher": [usher_colocate(occupancy[p["victim"]], occupancy[p["corunner"]]) for p in pairs],
        "orion": [orion_colocate(cls[p["victim"]], cls[p["corunner"]]) for p in pairs],
        "mlp": [p["mlp"] <= bound for p in pairs],
        "baseline": [p["baseline"] <= bound for p in pairs],
    }


def evaluate(pairs, kernel_info, occupancy, peaks, bounds=BOUNDS) -> dict:
    """Every rule scored at every bound, plus the per-kernel inputs of the two
    schedulers' rules."""
    measured = [p["measured"] for p in pairs]
    table = []
    for b in bounds:
        for rule, col in decisions(pairs, kernel_info, occupancy, peaks, b).items():
            table.append(dict(rule=rule, **score(col, measured, b)))
    kernels = {n: {"achieved_occupancy": round(occupancy[n], 4),
                   "arithmetic_intensity": round(k["flops"] / k["bytes"], 3) if k["bytes"] else None,
                   "orion_class": orion_class(k["flops"], k["bytes"], k["uses_tensor"], peaks)}
               for n, k in kernel_info.items()}
    return {"kernels": kernels, "scores": table}


def occupancy_by_kernel(order, captured) -> dict:
    """Match captured rows (launch order) to kernel names (the same order)."""
    if len(captured) != len(order):
        raise ValueError("occupancy capture has %d kernels, expected %d" % (len(captured), len(order)))
    return {n: v for n, (_k, v) in zip(order, captured)}


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) != 2:
        raise SystemExit(__doc__)
    with open(argv[0]) as f:
        c5 = json.loads(f.read().strip().splitlines()[-1])
    with open(argv[1]) as f:
        occ = occupancy_by_kernel(c5["kernels"], parse_ncu_occupancy(f.read()))
    out = evaluate(c5["pairs"], c5["kernel_info"], occ, c5["peaks"])
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
