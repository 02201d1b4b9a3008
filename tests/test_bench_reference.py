"""The bench's reference arm (the FP64 oracle on the host cores) runs on a
CPU-only machine and prints one JSON line with the contract's keys; under a
two-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(cmd, env=None):
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env={**os.environ, **(env or {})})
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.startswith("{")]


def check_line(d):
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] >= 1 and d["config"]["workload"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_single_process():
    lines = run([sys.executable, "bench.py", "--impl", "reference", "--config", "3sat",
                 "--steps", "2", "--warmup", "3"])
    assert len(lines) == 1
    check_line(json.loads(lines[0]))


def test_reference_arm_two_ranks_prints_once():
    lines = run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                 "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port", "29613",
                 "bench.py", "--impl", "reference", "--config", "3sat", "--gpus", "2",
                 "--steps", "2", "--warmup", "3"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    check_line(d)
    assert d["n_gpus"] == 2
