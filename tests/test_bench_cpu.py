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
    v, src = bench.tf32_peak()
    assert v == pytest.approx(d["bf16_tflops_sustained"] * 1.1 / 2.25, rel=1e-12)   # nominal TF32 / BF16
    assert "sustained" in src


def test_denominators_fall_back_without_the_file(bench, monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == {"hbm_gbs": 6800.0, "src": "fallback"}
    v, src = bench.tf32_peak()
    assert v == pytest.approx(1700.0 * 1.1 / 2.25) and src.startswith("fallback")


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
