"""The bench's reference arm (the CPU oracle timed on a bounded sample) on
the CPU: one JSON line with the keys of the bench contract, and nothing
printed by ranks other than 0.  The sample is shrunk so the test is fast."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(steps=2, warmup=1):
    return argparse.Namespace(steps=steps, warmup=warmup)


def test_reference_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 20000)
    assert bench.run_reference(_args(), rank=0, world=1) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "Gkeys/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["scaling"] == "weak" and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["n_per_array"] == 20000 and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "20000" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 1000)
    assert bench.run_reference(_args(1, 0), rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
