"""Host-side pieces of bench.py that decide what its JSON line reports: the
clock summary taken from nvidia-smi samples, and the DRAM traffic figure that
is reported only while the kernel source still matches the profile it came
from."""
from __future__ import annotations

import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2055.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_slowdown():
    c = bench.Clocks(0)
    c.lines = ["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.Clocks(0).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_bytes(b"__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _profile(root, sha, traffic=123456):
    (root / "profiles" / "p.md").write_text(f"code_sha256_16: {sha}\ntraffic_bytes_per_launch: {traffic}\n")


def test_traffic_reported_while_the_code_matches(fake_root):
    _profile(fake_root, bench.code_digest(str(fake_root / "k.cu")))
    assert bench._traffic("k.cu", "p.md") == 123456
    # comments and layout are not code
    (fake_root / "k.cu").write_bytes(b"// the kernel\n__global__   void k()\n{ /* empty */ }\n")
    assert bench._traffic("k.cu", "p.md") == 123456


def test_traffic_dropped_once_the_code_changed(fake_root):
    _profile(fake_root, bench.code_digest(str(fake_root / "k.cu")))
    (fake_root / "k.cu").write_bytes(b"__global__ void k() { int x = 0; }\n")
    assert bench._traffic("k.cu", "p.md") is None


def test_code_digest_is_sha256_of_the_normalised_code(tmp_path):
    f = tmp_path / "a.cu"
    f.write_text("int a; // note\n/* block\n comment */ int  b;\n")
    assert bench.code_digest(str(f)) == hashlib.sha256(b"int a;int b;").hexdigest()[:16]


def test_traffic_missing_profile(fake_root):
    assert bench._traffic("k.cu", "absent.md") is None


def test_whole_job_value_uses_the_slowest_rank():
    assert bench.job_value(1000.0, 4, 2.0) == 2000.0
    assert bench.rank_graph_range(3, 512) == (1536, 512)
