"""Host-side arithmetic of bench.py's roofline objects and exp-apply byte counts, on synthetic region
timers (no GPU): the figures the JSON line reports are the algorithmic work divided by the event-timed
duration, against the peak the line names."""
import importlib.util
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_exp_apply_bytes_hand_values(bench):
    # d16384_k100, b = 16 (m = n = 700): bf16 H read by each of the two sweeps, 16384 * 700 * 2 B = 22,937,600 B
    # per sweep; X (FP32) read twice and Y written once, 3 * 16384 * 16 * 4 B = 3,145,728 B
    assert bench.exp_apply_bytes(16384, 700, 16) == 2 * 22_937_600 + 3_145_728 == 49_020_928
    # one-pass form: the factor read once (it stays in shared memory for the second sweep)
    assert bench.exp_apply_bytes(16384, 700, 16, one_pass=True) == 22_937_600 + 3_145_728 == 26_083_328
    # d65536_k200, b = 32 (m = n = 2000): 2 * 262,144,000 B of bf16 H plus 3 * 8,388,608 B of X and Y
    assert bench.exp_apply_bytes(65536, 2000, 32) == 549_453_824


def _regions(bench, **over):
    regions = {r: (0.0, 0) for r in bench.REGIONS}
    work = {r: (0.0, 0.0) for r in ("gram", "tn_f64", "nn_f64", "oz_gemm", "oz_kernel", "oz_tiled")}
    for k, v in over.items():
        kind, name = k.split("__")
        (regions if kind == "t" else work)[name] = v
    return {"regions": regions, "work": work}


PK = {"hbm": 6768.1, "bf16": 1865.7, "bf16_sustained": 1694.0, "source": "measured"}


def test_roofline_tensor_core_step(bench):
    # 20 launches of the split product in 2.0 ms carrying 12 GB of digit planes and results and 1e12 flops
    r = _regions(bench, t__oz_kernel=(2.0, 20), w__oz_kernel=(1e12, 12e9))
    rl = bench.roofline_of("d65536_k200", r, 1, "tc", PK)
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and rl["peak"] == PK["hbm"]
    assert rl["achieved"] == pytest.approx(6000.0)                # 12e9 B / 2e-3 s
    assert rl["frac"] == pytest.approx(6000.0 / 6768.1)
    assert rl["algorithmic_bytes_per_launch"] == pytest.approx(6e8)
    assert rl["avg_launch_us"] == pytest.approx(100.0)
    assert rl["launches"] == 20
    assert rl["tensor_tflops_bf16"] == pytest.approx(500.0)       # 1e12 flops / 2e-3 s
    assert rl["traffic"] == bench.OZ_TRAFFIC_BYTES["d65536_k200"]
    assert "measured" in rl["peak_source"]
    # a workload without an ncu capture reports no traffic
    assert bench.roofline_of("d4096_k40", r, 1, "tc", PK)["traffic"] is None


def test_roofline_fp64_step_counts_one_triangle(bench):
    d, n = 65536, 2000
    flops = d * n * (n + 1)                                       # SYRK: one triangle of G_W
    r = _regions(bench, t__gram=(200.0, 1), w__gram=(float(flops), 8.0 * d * n))
    rl = bench.roofline_of("d65536_k200", r, 1, "f64", PK)
    assert rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    assert rl["achieved"] == pytest.approx(flops / 0.2 / 1e12)
    assert rl["frac"] == pytest.approx(flops / 0.2 / 1e12 / bench.NOMINAL_FP64_TFLOPS)
    assert rl["flops_per_launch"] == pytest.approx(flops)
    assert rl["peak"] == bench.NOMINAL_FP64_TFLOPS


def test_roofline_without_launches_is_not_a_number(bench):
    rl = bench.roofline_of("d65536_k200", _regions(bench), 1, "tc", PK)
    assert math.isnan(rl["achieved"]) and rl["launches"] == 0
