"""Host arithmetic of bench.py's attribute-stage rooflines (no GPU): work per symbol, units
and peaks, checked against numbers worked by hand."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


PK = {"hbm_gbs": 6500.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2000.0}


def test_static_attributes_hbm(bench):
    r = bench.attr_roofline(1, 1000, 40_000, 0.001, PK)  # 1 us for 1,000 Gaussians
    assert r["bound"] == "hbm" and r["algorithmic_bytes"] == 40_000 + 4 * 56 * 1000
    assert r["achieved"] == pytest.approx(264_000 / 1e-6 / 1e9) and r["frac"] == pytest.approx(r["achieved"] / 6500)


def test_learned_alu_and_tensor(bench):
    r = bench.attr_roofline(2, 1000, 0, 1.0, PK)  # 1 ms
    assert r["bound"] == "alu" and r["algorithmic_ops"] == 10 * 256 * 56 * 1000
    assert r["peak"] == pytest.approx(148 * 128 * 2.0)  # Gop/s at 2 GHz
    assert r["achieved"] == pytest.approx(143.36)  # 143.36 M ops in 1 ms
    assert r["tensor"]["achieved"] == pytest.approx(2 * 20480 * 56_000 / 1e-3 / 1e12)


def test_position_aware_tensor(bench):
    r = bench.attr_roofline(3, 1000, 0, 1.0, PK)
    assert r["algorithmic_flops"] == 2 * 4480 * 56_000 + 2 * 4800 * 1000
    assert r["unit"] == "TFLOP/s" and r["frac"] == pytest.approx(r["achieved"] / 1800)
    assert bench.attr_roofline(3, 1000, 0, 1.0, {})["peak_source"] == "fallback 1800"


def test_reference_arm_line_contract():
    """bench.py --impl reference prints one JSON line with the contract's keys: the oracle's
    throughput, its cpu_baseline description and an e2e block with no host-device bytes."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gaussians/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gaussians/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n_rows"] == 18_000
