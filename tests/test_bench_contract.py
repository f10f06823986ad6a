"""CPU tests of the benchmark's reference arm (`bench.py --impl reference`).

The reference arm times the FP64 oracle decoder on the host cores over a
bounded sample of the workload.  These tests run it on the 400-signal mixed
workload with a short sample and check the JSON line it prints against the
benchmark's contract: one line, the metric and unit of the product arm,
`impl: reference`, a `cpu_baseline` that describes this run and an `e2e` with
no host-device traffic.  They also check that the arm keeps out of the product:
neither the library (`libfptc.so`) nor torch is loaded in its process, and a
rank other than 0 of a multi-process launch prints nothing and exits 0.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = """
import sys
sys.argv = ["bench.py"] + sys.argv[1:]
import bench
rc = bench.main()
maps = open("/proc/self/maps").read() if sys.platform.startswith("linux") else ""
print("MAPPED", int("libfptc" in maps), int("torch" in sys.modules), flush=True)
sys.exit(rc or 0)
"""


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, "-c", _RUN, *args], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


@pytest.fixture(scope="module")
def reference_run():
    r = _run(["--impl", "reference", "--workload", "mixed_small", "--steps", "2", "--warmup", "3",
              "--ref-seconds", "0.3"])
    assert r.returncode == 0, r.stderr[-2000:]
    return r


def test_reference_arm_prints_one_contract_line(reference_run):
    lines = [ln for ln in reference_run.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "decoded GB/s (float32 out)" and d["unit"] == "GB/s"
    assert d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["vs_baseline"] is None
    cfg = d["config"]
    assert cfg["workload"] == "mixed_400_logu_4096_262144" and cfg["n_streams"] == 400
    assert cfg["out_bytes"] == 4 * cfg["n_samples"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["unit"] == "GB/s" and cb["value"] == d["value"]
    assert cb["cores"] >= 1 and "streams" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_loads_neither_library_nor_torch(reference_run):
    marks = [ln for ln in reference_run.stdout.splitlines() if ln.startswith("MAPPED")]
    assert marks == ["MAPPED 0 0"]


def test_reference_arm_other_ranks_do_no_work():
    r = _run(["--impl", "reference", "--workload", "mixed_small", "--steps", "1", "--warmup", "3"],
             {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_warmup_below_three_is_refused():
    r = _run(["--impl", "reference", "--workload", "mixed_small", "--steps", "1", "--warmup", "2"])
    assert r.returncode != 0
    assert "--warmup must be >= 3" in r.stderr
