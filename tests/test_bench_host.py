"""Host logic of bench.py on CPU: the clock record taken during the timed
region, and the rule that a kernel's DRAM traffic is reported only while
the kernel sources are the ones the ncu summary was taken on."""
import os

import bench


def _summary_of(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(l + "\n" for l in lines))
    s = bench.ClockSampler(0)
    s.path = str(path)
    return s.summary()


def test_clock_record_median_max_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "malformed line",
    ]
    d = _summary_of(tmp_path, rows)
    assert d["samples"] == 3
    assert d["sm_mhz"] == 2070.0 and d["sm_max_mhz"] == 2070.0
    assert d["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")  # the record is consumed


def test_clock_record_flags_thermal_and_hw_slowdown(tmp_path):
    rows = [
        "0, 1500, 2070, 1000.0, 0x48, Active, Not Active, Active, Not Active",
        "0, 1600, 2070, 1000.0, 0x20, Not Active, Active, Not Active, Not Active",
    ]
    d = _summary_of(tmp_path, rows)
    assert d["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert d["sm_mhz"] == 1550.0


def test_clock_record_without_samples(tmp_path):
    assert _summary_of(tmp_path, [])["reasons"] == ["no samples"]


def test_traffic_reported_only_for_the_profiled_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = bench.kernel_source_hash()
    (prof / "dram_traffic.md").write_text(
        "| kernel | sources hash | bytes per launch |\n|---|---|---|\n"
        f"| bead_kernel | {src} | 176505344 |\n| z_spectral | 0123456789ab | 16876288 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: src)
    assert bench.profiled_traffic("bead_kernel") == 176505344
    assert bench.profiled_traffic("z_spectral") is None  # taken on other sources
    assert bench.profiled_traffic("xy_forward_plane") is None  # not profiled


def test_kernel_source_hash_changes_with_any_kernel_source(tmp_path, monkeypatch):
    import shutil

    src = os.path.join(bench.ROOT, "paper_2302_02474_gb300", "csrc")
    dst = tmp_path / "paper_2302_02474_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash() and len(h0) == 12
    for name in sorted(os.listdir(dst)):
        if name.endswith((".cu", ".cuh", ".h")):
            f = dst / name
            text = f.read_text()
            f.write_text(text + "\n")
            assert bench.kernel_source_hash() != h0, name
            f.write_text(text)
    assert bench.kernel_source_hash() == h0
