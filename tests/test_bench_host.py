"""Host-side pieces of bench.py that need no GPU: the clock-sample parser
behind the JSON line's `clocks` (whose throttle reasons reject a run), and
the lookup of the committed ncu traffic, which must refuse a summary taken
on other kernel source."""
import os
import subprocess
import sys

import bench


def sample(sm, mx, *reasons):
    flags = ["Active" if r else "Not Active" for r in reasons]
    return "0, %s, %s, 812.5, 0x0000000000000004, %s\n" % (sm, mx, ", ".join(flags))


def test_clock_parser_takes_median_max_and_reasons():
    lines = [sample(2070, 2070, False, False, False, False),
             sample(1980, 2070, False, False, False, True),
             sample(2070, 2070, False, False, False, False),
             "garbage line\n",
             "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active\n"]
    out = bench.Clocks.parse(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_parser_reports_every_throttle_reason_and_empty_input():
    lines = [sample(1500, 2070, True, False, False, False), sample(1400, 2070, False, True, True, False)]
    out = bench.Clocks.parse(lines)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450.0
    assert bench.Clocks.parse([]) is None
    assert bench.Clocks.parse(["0, 1, 2\n"]) is None


def test_profiled_traffic_requires_the_current_kernel_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    text = "kernel source hash: %s\ndram bytes per launch (read+write): 12345678\n"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash",
                        lambda precision="fp64": {"fp64": "abcdef0123456789", "fp32": "0123456789abcdef"}[precision])
    (prof / "nbjm_sweep_w.md").write_text(text % "abcdef0123456789")
    assert bench.profiled_traffic("w") == 12345678.0
    (prof / "nbjm_sweep_w.md").write_text(text % "0000000000000000")
    assert bench.profiled_traffic("w") is None
    assert bench.profiled_traffic("missing") is None
    # the FP32 summary is keyed on the FP32 sweeps' own sources
    (prof / "nbjm_sweep_f32_w.md").write_text(text % "0123456789abcdef")
    assert bench.profiled_traffic("w", "fp32") == 12345678.0
    (prof / "nbjm_sweep_f32_w.md").write_text(text % "abcdef0123456789")
    assert bench.profiled_traffic("w", "fp32") is None


def test_profiled_traffic_requires_the_same_kernel(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda precision="fp64": "abcdef0123456789")
    one = bench.sweep_kernel_name({"threads": 64, "steps_per_lane": 0, "two_ended": 0}, "double")
    two = bench.sweep_kernel_name({"threads": 64, "steps_per_lane": 0, "two_ended": 1}, "double")
    bulk = bench.sweep_kernel_name({"threads": 128, "steps_per_lane": 2, "two_ended": 1}, "float")
    assert len({one, two, bulk}) == 3 and "twisted" in two and "bulk" in bulk
    (prof / "nbjm_sweep_w.md").write_text("kernel source hash: abcdef0123456789\nprofiled kernel: %s\n"
                                          "dram bytes per launch (read+write): 42\n" % one)
    assert bench.profiled_traffic("w", "fp64", one) == 42.0
    assert bench.profiled_traffic("w", "fp64", two) is None
    assert bench.profiled_traffic("w", "fp64") == 42.0


def test_kernel_hash_covers_the_sweep_sources():
    for precision in ("fp64", "fp32"):
        h = bench.kernel_source_hash(precision)
        assert len(h) == 16 and int(h, 16) >= 0
        for name in bench.KERNEL_SOURCES[precision]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2304_04980_gb300", "csrc", name))
    assert bench.kernel_source_hash("fp64") != bench.kernel_source_hash("fp32")


def test_clock_stop_ends_the_sampler_and_parses_its_file(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text(sample(2070, 2070, False, False, False, False) * 2)
    c = bench.Clocks()
    c.path = str(path)
    c.proc = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(60)"])
    out = c.stop()
    assert c.proc.poll() is not None
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 2}
    assert not path.exists()
    assert bench.Clocks().stop() is None
