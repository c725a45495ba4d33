"""bench.py on a machine without a GPU: the reference arm (the CPU oracle on
a bounded sample of the sweep) prints its one JSON line, also under a
two-rank launch where rank 0 alone runs; the main arm fails instead of
falling back to the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def check_reference_line(d, n_gpus):
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus
    assert d["unit"] == "schemes/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "d7_batched_sweep"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "schemes/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_one_line():
    p = subprocess.run([sys.executable, BENCH, "--impl", "reference", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
    assert p.returncode == 0, p.stdout[-2000:]
    lines = json_lines(p.stdout)
    assert len(lines) == 1, p.stdout[-2000:]
    check_reference_line(lines[0], 1)


def test_reference_arm_under_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           BENCH, "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stdout[-2000:]
    lines = json_lines(p.stdout)
    assert len(lines) == 1, p.stdout[-2000:]
    check_reference_line(lines[0], 2)


def test_main_arm_has_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = subprocess.run([sys.executable, BENCH, "--steps", "3", "--warmup", "3"], cwd=ROOT,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
    assert p.returncode != 0
    assert not [d for d in json_lines(p.stdout) if "value" in d]
