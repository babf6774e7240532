"""The reference arm of bench.py on the CPU: its JSON line carries every key
of the benchmark contract (with the oracle's timing stubbed out), and the
oracle sampling itself runs on a small set."""
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
    stub = {"value": 0.5, "unit": bench.UNIT, "cores": 4, "kind": "oracle", "sample": "stub",
            "seconds_per_set": 2.0}
    monkeypatch.setattr(bench, "oracle_sample", lambda inputs, n, count_n=256: dict(stub))
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    required = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"}
    assert required <= set(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 0.5 and line["ms_per_step"] == 2000.0 and line["higher_is_better"]
    assert (line["steps"], line["warmup"], line["n_gpus"]) == (2, 3, 1)
    assert line["e2e"] == {"value": 0.5, "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert set(line["cpu_baseline"]) == {"value", "unit", "cores", "kind", "sample"}
    assert line["config"]["grid"] == [16, 16, 16]


def test_reference_arm_other_ranks_print_nothing(monkeypatch, capsys):
    bench, args = _args(monkeypatch, ["--impl", "reference", "--n", "16"])
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_oracle_sample_times_the_oracle_on_a_small_set():
    sys.path.insert(0, ROOT)
    import bench

    res = bench.oracle_sample(bench.workload(16), 16, count_n=16)
    assert res["kind"] == "oracle" and res["cores"] >= 1 and res["unit"] == bench.UNIT
    assert res["value"] > 0 and abs(res["value"] * res["seconds_per_set"] - 1.0) < 1e-12
    assert "V(2,2)" in res["sample"] and "16^3" in res["sample"]
