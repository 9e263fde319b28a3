"""bench.py runs end to end on the GPU (a short run of each workload mode) and prints the contract's keys."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "clocks", "gpu_launches", "e2e", "roofline"}


def _run(*args):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert KEYS <= set(line), KEYS - set(line)
    assert line["value"] > 0 and line["gpu_launches"] > 0
    assert set(line["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    return line


def test_bench_default_workload_short():
    _run("--steps", "3", "--warmup", "3", "--no-cpu-baseline", "--no-exp-apply")


def test_bench_batched_workload_short():
    _run("--workload", "batched64", "--steps", "1", "--warmup", "1", "--no-cpu-baseline")
