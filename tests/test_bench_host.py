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
