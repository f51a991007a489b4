"""The reference arm of the benchmark on CPU: `bench.py --impl reference` times
the oracle (the only CPU program of the method) and prints one JSON line in the
benchmark's format.  Run here at R-MAT scale 14 so that it takes a second."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *extra],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_line_has_the_benchmark_format():
    d = _run("--scale", "14", "--steps", "2", "--warmup", "1")
    assert d["impl"] == "reference"
    assert d["unit"] == "GTEPS" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # value = m / step time
    m = d["config"]["m"]
    assert abs(d["value"] - m / (d["ms_per_step"] / 1e3) / 1e9) <= 1e-9 * max(1.0, d["value"])
    assert d["dtype"] == "int32" and d["data"] == "synthetic" and d["vs_baseline"] is None
    # the config names the scale that ran
    assert d["config"]["scale"] == 14 and "scale 14" in d["config"]["workload"]
    assert d["same_config"] is True
    assert d["config"]["n"] == 1 << 14
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] == (os.cpu_count() or 1) and "scale 14" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert 0 < d["cut"] < m and d["maxbw"] <= d["lmax"]


def test_reference_result_does_not_depend_on_the_step_count():
    a = _run("--scale", "14", "--steps", "1", "--warmup", "0")
    b = _run("--scale", "14", "--steps", "2", "--warmup", "1")
    assert (a["cut"], a["maxbw"], a["lmax"]) == (b["cut"], b["maxbw"], b["lmax"])
