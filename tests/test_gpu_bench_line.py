"""The benchmark's default line on a small case: the plain workload at 2^20
keys per array, in its default form (four host threads, one context and
stream each) and from one thread on one stream.  Checks the keys of the
bench contract and that both forms report a positive throughput."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*extra):
    r = subprocess.run([sys.executable, "bench.py", "--n", str(1 << 20), "--steps", "2",
                        "--warmup", "3", "--no-cpu-baseline", *extra],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _common(d):
    assert d["metric"] == "sorted Gkeys/s" and d["unit"] == "Gkeys/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 3, 1)
    assert d["config"]["n_per_array"] == 1 << 20 and d["config"]["arrays_per_step"] == 4
    assert d["gpu_launches"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 8 * 4 << 20
    assert "sm_mhz" in d["clocks"]


def test_default_line_four_threads():
    d = _line()
    _common(d)
    assert d["config"]["sort_threads"] == 4
    seq = d["sequential"]
    assert seq["value"] > 0 and seq["ms_per_step"] > 0 and seq["unit"] == "Gkeys/s"


def test_one_stream_line():
    d = _line("--sort-threads", "1")
    _common(d)
    assert d["config"]["sort_threads"] == 1
    assert "sequential" not in d
