"""Host logic of the pairing rules (Sec. 3 Pitfalls 1 and 2) on hand-made inputs: the
two pitfall examples of the paper come out as violations of the rule they refute,
and the scores are counted by hand."""
import pytest

from paper_2501_16909_b300 import pairing as PG

PEAKS = {"tensor": 1.8e15, "fp32": 77e12, "hbm": 6.4e12}  # ridges: 281.25 and 12.03 flop/B

NCU_CSV = """==WARNING== Note: Running with unmodified GPU clocks.
==PROF== Connected to process 1 (/usr/bin/python3)
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"1","7","python3","h","void <unnamed>::softmax_kernel<256>(const float *, float *, long, long)","1","13","(256, 1, 1)","(592, 1, 1)","0","10.3","Command line profiler metrics","sm__warps_active.avg.pct_of_peak_sustained_active","%","48.50"
"0","7","python3","h","void <unnamed>::gemm_bf16_kernel<256, 3>(CUtensorMap, CUtensorMap, float *)","1","13","(192, 1, 1)","(148, 1, 1)","0","10.3","Command line profiler metrics","sm__warps_active.avg.pct_of_peak_sustained_active","%","9.37"
==PROF== Disconnected from process 1
"""


def test_usher_rule_is_a_strict_sum_below_one():
    assert PG.usher_colocate(0.0625, 0.0625)
    assert PG.usher_colocate(0.3, 0.6)
    assert not PG.usher_colocate(0.5, 0.5)
    assert not PG.usher_colocate(0.7, 0.4)


def test_orion_class_uses_the_ridge_of_the_kernels_pipe():
    # exactly at the fp32 ridge (77e12 / 6.4e12 flop per byte) counts as compute-bound
    assert PG.orion_class(77e12, 6.4e12, False, PEAKS) == "compute"
    assert PG.orion_class(77e12, 6.5e12, False, PEAKS) == "memory"
    # a GEMM at 128 flop/B is compute-bound on the fp32 ridge but memory-bound on the tensor ridge
    assert PG.orion_class(128.0, 1.0, False, PEAKS) == "compute"
    assert PG.orion_class(128.0, 1.0, True, PEAKS) == "memory"
    assert PG.orion_class(1.0, 0.0, True, PEAKS) == "compute"
    assert PG.orion_colocate("compute", "memory") and not PG.orion_colocate("memory", "memory")


def test_score_counts_by_hand():
    s = PG.score([True, True, False, False], [1.05, 1.3, 2.0, 1.1], 1.25)
    assert (s["colocated"], s["violations"], s["missed"], s["within_bound"]) == (2, 1, 1, 2)
    assert s["precision"] == 0.5 and s["recall"] == 0.5 and s["worst_colocated"] == 1.3
    none = PG.score([False, False], [1.0, 3.0], 1.5)
    assert none["colocated"] == 0 and none["precision"] is None and none["worst_colocated"] is None
    assert none["missed"] == 1 and none["recall"] == 0.0


def test_pitfall_examples_are_violations_of_the_rules_they_refute():
    # Pitfall 1: two fp32 compute kernels at 6.25 % achieved occupancy each slow each
    # other down 1.73x; Pitfall 2: a compute kernel and a copy kernel, the copy 2x slower
    kernels = {
        "compute_a": {"flops": 1e12, "bytes": 1e6, "uses_tensor": False},
        "compute_b": {"flops": 1e12, "bytes": 1e6, "uses_tensor": False},
        "copy": {"flops": 0.0, "bytes": 1e9, "uses_tensor": False},
    }
    occ = {"compute_a": 0.0625, "compute_b": 0.0625, "copy": 0.5}
    pairs = [
        {"victim": "compute_a", "corunner": "compute_b", "measured": 1.73, "mlp": 1.7, "baseline": 1.0},
        {"victim": "copy", "corunner": "compute_a", "measured": 2.0, "mlp": 1.9, "baseline": 1.1},
    ]
    res = PG.evaluate(pairs, kernels, occ, PEAKS, bounds=(1.25,))
    by = {r["rule"]: r for r in res["scores"]}
    assert by["usher"]["colocated"] == 2 and by["usher"]["violations"] == 2
    assert by["orion"]["colocated"] == 1 and by["orion"]["violations"] == 1
    assert by["mlp"]["colocated"] == 0 and by["mlp"]["violations"] == 0
    assert by["baseline"]["violations"] == 2
    assert res["kernels"]["copy"]["orion_class"] == "memory"
    assert res["kernels"]["compute_a"]["orion_class"] == "compute"
    assert len(res["scores"]) == 4


def test_ncu_csv_rows_in_launch_order(tmp_path):
    rows = PG.parse_ncu_occupancy(NCU_CSV)
    assert [n.split("::")[1].split("<")[0] for n, _ in rows] == ["gemm_bf16_kernel", "softmax_kernel"]
    assert rows[0][1] == pytest.approx(0.0937) and rows[1][1] == pytest.approx(0.485)
    occ = PG.occupancy_by_kernel(["decode.qkv", "decode.softmax"], rows)
    assert occ == {"decode.qkv": pytest.approx(0.0937), "decode.softmax": pytest.approx(0.485)}
    with pytest.raises(ValueError):
        PG.occupancy_by_kernel(["one"], rows)


def test_cli_rescoring_of_a_saved_result(tmp_path, capsys):
    c5 = {"kernels": ["decode.qkv", "decode.softmax"],
          "kernel_info": {"decode.qkv": {"flops": 4.0e9, "bytes": 3.2e7, "uses_tensor": True},
                          "decode.softmax": {"flops": 4.0e7, "bytes": 6.7e7, "uses_tensor": False}},
          "peaks": PEAKS,
          "pairs": [{"victim": "decode.softmax", "corunner": "decode.qkv", "measured": 1.2, "mlp": 1.3,
                     "baseline": 1.1}]}
    (tmp_path / "c5.json").write_text("log line\n" + __import__("json").dumps(c5) + "\n")
    (tmp_path / "occ.csv").write_text(NCU_CSV)
    out = PG.main([str(tmp_path / "c5.json"), str(tmp_path / "occ.csv")])
    assert len(out["scores"]) == 4 * len(PG.BOUNDS)
    usher = [r for r in out["scores"] if r["rule"] == "usher"]
    assert all(r["colocated"] == 1 for r in usher)  # 0.094 + 0.485 < 1
    orion = [r for r in out["scores"] if r["rule"] == "orion"]
    assert all(r["colocated"] == 0 for r in orion)  # both memory-bound (125 flop/B under the tensor ridge)
