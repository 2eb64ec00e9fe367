"""Host-side pieces of bench.py: the clock record and the DRAM-traffic lookup."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary(bench):
    na, act = "Not Active", "Active"
    lines = [
        f"0, 2070, 2070, 800.1, 0x0, {na}, {na}, {na}, {na}\n",
        f"0, 1950, 2070, 1390.5, 0x4, {na}, {na}, {na}, {act}\n",
        f"0, 2070, 2070, 1200.0, 0x0, {na}, {na}, {na}, {na}\n",
        "garbage line\n",
    ]
    c = bench.Clocks.summarize(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.Clocks.summarize([f"0, 1500, 2070, 900, 0x8, {na}, {act}, {na}, {na}\n"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.Clocks.summarize([])["reasons"] == ["no samples"]


def test_traffic_only_for_the_sources_it_was_taken_on(bench, tmp_path, monkeypatch):
    from paper_2501_02747_gb300 import build
    (tmp_path / "profiles").mkdir()
    f = tmp_path / "profiles" / "traffic_k_demo.txt"
    f.write_text("# comment: with a colon\ndram_bytes_per_launch: 12345\n"
                 f"source_digest: {build._digest()}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_demo") == 12345.0
    f.write_text("dram_bytes_per_launch: 12345\nsource_digest: 0123\n")
    assert bench.traffic_from_profiles("k_demo") is None       # other sources
    assert bench.traffic_from_profiles("k_missing") is None
