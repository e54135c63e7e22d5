"""CPU checks of bench.py's reference arm (the CPU oracle, timed on the host
cores): one JSON line with the contract's keys, alone and under torchrun
with two ranks (rank 0 alone prints)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.timeout(600, method="thread")


def _lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check(line):
    assert line["impl"] == "reference" and line["metric"] == "decompressed GB/s" and line["unit"] == "GB/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] >= 1
    assert line["warmup"] >= 3 and line["steps"] >= 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e = line["e2e"]
    assert e["value"] == line["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("csv1g")
    assert line["config"]["bytes_per_stream"] == 1 << 30 and line["config"]["parallelism"].startswith("replicas")


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-blocks", "1", "--ref-pool", str(8 << 20)], cwd=ROOT, capture_output=True, text=True, timeout=500)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0])


def test_reference_arm_under_torchrun_prints_once():
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29571", "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-blocks", "1",
                        "--ref-pool", str(8 << 20)],
                       cwd=ROOT, capture_output=True, text=True, timeout=500)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0])


def test_launches_in_flight_from_spans():
    """The serving line's overlap figure: launches in flight at once, from
    each distinct launch's (start, completion) host times."""
    import bench
    c = bench._concurrency({(0.0, 2.0), (1.0, 3.0), (2.5, 4.0), (5.0, 6.0)})
    assert c == {"launches": 4, "max": 2, "mean": 1.3}
    assert bench._concurrency(set()) == {"launches": 0, "max": 0, "mean": 0.0}
    # one launch at a time, back to back
    assert bench._concurrency({(0.0, 1.0), (1.0, 2.0)})["max"] == 1
