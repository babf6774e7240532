"""Host logic of bench.py on the CPU: the reference arm's JSON line carries
every key of the benchmark contract (with the oracle's timing stubbed out),
whole oracle solve sets are timed within the budget, and the roofline object follows its
definition (dominant fine-level class, algorithmic bytes per launch over the
average launch time, measured peak, traffic scaled from the committed capture
and null once the kernel source changed)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(monkeypatch, argv):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    return bench, bench.parse()


def test_reference_line_carries_the_contract(monkeypatch, capsys):
    bench, args = _args(monkeypatch, ["--impl", "reference", "--n", "16", "--steps", "2",
                                      "--warmup", "3"])
    info = [(14, 9e-11), (10, 8e-11), (8, 7e-11), (3, 6e-11)]
    monkeypatch.setattr(bench, "oracle_sets",
                        lambda inputs, n, max_sets, budget: (2.0, 2, list(info), 4))
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    required = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"}
    assert required <= set(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 0.5 and line["ms_per_step"] == 2000.0 and line["higher_is_better"]
    # the steps that ran (whole oracle sets), the requested counts beside them
    assert (line["steps"], line["warmup"], line["n_gpus"]) == (2, 0, 1)
    assert (line["steps_requested"], line["warmup_requested"]) == (2, 3)
    assert line["e2e"] == {"value": 0.5, "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert set(line["cpu_baseline"]) == {"value", "unit", "cores", "kind", "sample"}
    assert line["cpu_baseline"]["cores"] == 4 and line["cpu_baseline"]["value"] == 0.5
    # the config describes the CPU oracle, not the GPU run
    cfg = line["config"]
    assert cfg["grid"] == [16, 16, 16] and cfg["precision"] == "fp64"
    assert "oracle" in cfg["implementation"] and "concurrency" not in cfg


def test_oracle_sets_stop_within_the_budget(monkeypatch):
    """Whole sets run until the requested count, or until the next one would
    end after the budget; at least one always runs."""
    sys.path.insert(0, ROOT)
    import bench

    clock = [0.0]
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock[0])

    def fake_set(inputs, n):
        clock[0] += 30.0
        return 30.0, [(5, 1e-11)] * 4

    monkeypatch.setattr(bench, "oracle_set", fake_set)
    sec, nsets, info, _ = bench.oracle_sets(None, 16, max_sets=20, budget_s=100.0)
    assert (sec, nsets) == (30.0, 3)  # a fourth set would end at 120 s
    sec, nsets, _, _ = bench.oracle_sets(None, 16, max_sets=2, budget_s=1000.0)
    assert nsets == 2
    sec, nsets, _, _ = bench.oracle_sets(None, 16, max_sets=5, budget_s=1.0)
    assert nsets == 1


def test_reference_arm_other_ranks_print_nothing(monkeypatch, capsys):
    bench, args = _args(monkeypatch, ["--impl", "reference", "--n", "16"])
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_oracle_baseline_times_whole_solves_on_a_small_set():
    sys.path.insert(0, ROOT)
    import bench

    res = bench.oracle_baseline(bench.workload(16), 16)
    assert res["kind"] == "oracle" and res["cores"] >= 1 and res["unit"] == bench.UNIT
    assert res["value"] > 0 and abs(res["value"] * res["seconds_per_set"] - 1.0) < 1e-12
    assert res["sets"] == 1 and len(res["cycles"]) == 4 and min(res["cycles"]) >= 1
    assert max(res["rel_resid"]) <= bench.TOL
    assert "whole solve set" in res["sample"] and "16^3" in res["sample"]


def _prof():
    return {"smooth": {"ms": 100.0, "launches": 500, "bytes": 500 * 969.0e6},
            "resid64": {"ms": 50.0, "launches": 20, "bytes": 20 * 4.3e9},
            "coarse": {"ms": 40.0, "launches": 1000, "bytes": 0.0}}


def test_roofline_of_the_dominant_class():
    sys.path.insert(0, ROOT)
    import bench

    pk, src = bench.peaks()
    r = bench.roofline(_prof(), _prof(), 512)
    assert r["kernel"] == "smooth" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    achieved = 969.0e6 / (0.2e-3) / 1e9          # bytes per launch over 0.2 ms per launch
    assert abs(r["achieved"] - round(achieved, 1)) < 1e-9
    assert r["peak"] == float(pk["hbm_gbs"])
    assert abs(r["frac"] - round(achieved / float(pk["hbm_gbs"]), 4)) < 1e-12
    assert abs(sum(r["class_share"].values()) - 1.0) < 1e-3
    assert "coarse" not in r["class_gbs"] and set(r["class_gbs"]) == {"smooth", "resid64"}
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        ent = json.load(fh)["smooth"]
    if ent["source_hash"] == bench.source_hash(bench.KERNEL_SOURCES["smooth"]):
        assert r["traffic"] == round(ent["dram_over_algorithmic"] * 969.0e6)
    else:
        assert r["traffic"] is None


def test_traffic_is_null_once_the_kernel_source_changed(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setitem(bench.KERNEL_SOURCES, "smooth", ["bench.py"])  # another file's hash
    assert bench.traffic_for("smooth", 1e9) is None
    assert bench.traffic_for("no-such-class", 1e9) is None


def test_roofline_needs_a_fine_level_class_and_peaks_fall_back(monkeypatch, tmp_path):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.roofline({"coarse": {"ms": 5.0, "launches": 10, "bytes": 0.0}}, {}, 512) is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))  # no MEASURED_PEAKS.json there
    pk, src = bench.peaks()
    assert src == "fallback" and pk["hbm_gbs"] == 6800.0
