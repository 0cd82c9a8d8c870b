"""Host logic of bench.py's roofline fields, on the CPU: the HBM and TF32 denominators (the
measured peaks, or the fallback when the measurement file is absent) and the `traffic` figure,
which is reported only while the kernel source is the one the ncu summary was captured from."""
import hashlib
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_denominators_are_the_measured_peaks(bench):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks in this checkout")
    d = json.load(open(path))
    assert bench.peaks() == {"hbm_gbs": d["hbm_gbs"], "src": "measured"}
    v, src, recipe = bench.tf32_peak()
    # the measured per-SM kind::tf32 rate (4096 flop/cycle/SM) x 152 SMs x the maximum clock
    assert v == pytest.approx(4096 * 152 * d["sm_max_mhz"] * 1e6 / 1e12, rel=1e-12)
    assert recipe == pytest.approx(d["bf16_tflops_sustained"] * 1.1 / 2.25, rel=1e-12)   # nominal TF32 / BF16
    v2, src2, _ = bench.tf32_peak(1500.0)                  # the clock sampled during the run
    assert v2 == pytest.approx(4096 * 152 * 1500e6 / 1e12) and "1500 MHz" in src2


def test_denominators_fall_back_without_the_file(bench, monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == {"hbm_gbs": 6800.0, "src": "fallback"}
    v, src, recipe = bench.tf32_peak()
    assert v == pytest.approx(4096 * 152 * 2070e6 / 1e12) and recipe == pytest.approx(1700.0 * 1.1 / 2.25)


def test_traffic_only_for_the_captured_source(bench, monkeypatch, tmp_path):
    csrc = tmp_path / "paper_1807_04180_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = csrc / "solve.cu"
    src.write_bytes(b"// kernel source at capture\n")
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "k_solve2d_2d_heterogeneous_1024.md"
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    prof.write_text(f"# summary\n\n    source_sha1: {sha}\n    precision: mixed\n"
                    "    traffic_bytes_per_launch: 2852013712\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.solve_traffic("mixed") == 2852013712
    assert bench.solve_traffic("fp64") is None           # captured in another precision
    src.write_bytes(b"// kernel source edited since\n")
    assert bench.solve_traffic("mixed") is None          # stale once the source changes
    prof.unlink()
    assert bench.solve_traffic("mixed") is None
