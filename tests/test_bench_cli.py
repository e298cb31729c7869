"""The benchmark's command-line contract, on the CPU: the reference arm (the FP64 oracle
timed on the host cores) prints one JSON line with the keys the contract names, and the
argument checks reject what the timing rules forbid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=300, cwd=ROOT)


def test_reference_arm_line():
    r = _run("--impl", "reference", "--workload", "plain_small", "--steps", "3", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "plain_small"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_too_few_warmup_steps_rejected():
    r = _run("--impl", "reference", "--workload", "plain_small", "--steps", "3", "--warmup", "2")
    assert r.returncode != 0
    assert "warmup" in r.stderr


def test_workloads_listed():
    r = _run("--help")
    assert r.returncode == 0
    for w in ("plain_large", "plain_small", "precision_large", "batched", "unrolled"):
        assert w in r.stdout
