"""The bench's clock record (what makes a measured number acceptable): nvidia-smi samples taken
during the timed region are reduced to the median SM clock, the maximum clock and the throttle
reasons seen.  A fake nvidia-smi on PATH stands in for the GPU."""
import os
import stat
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_summary_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2050, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(lines).summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_summary_flags_thermal_and_hw_slowdown():
    lines = ["1500, 2070, 1300, 0x48, Active, Not Active, Active, Not Active"] * 3
    out = _sampler(lines).summary()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_summary_without_samples():
    assert _sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_sampler_reads_a_running_nvidia_smi(tmp_path, monkeypatch):
    """The sampler starts nvidia-smi with the query and a 100 ms period and collects its lines."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo \"$@\" > \"$(dirname \"$0\")/args.txt\"\n"
                    "i=0\nwhile [ $i -lt 50 ]; do\n"
                    "  echo '2070, 2070, 1000, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "  i=$((i+1)); sleep 0.02\ndone\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    with bench.ClockSampler(3) as clk:
        pass
    out = clk.summary()
    assert out["samples"] >= 1 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    args = (tmp_path / "args.txt").read_text()
    assert "-i 3" in args and "--query-gpu=" in args and "-lms 100" in args


def test_traffic_is_reported_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    """`roofline.traffic` comes from the committed ncu summary only while the hash of the kernel
    code it records (comments excluded) matches the current sources."""
    import json
    import shutil

    for rel in bench.PASS_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    path = tmp_path / "profiles" / "defer_kernel_image8192_f64_traffic.json"
    path.write_text(json.dumps({"source_hash": bench.pass_kernel_hash(), "dram_bytes_per_launch": 1.0}))
    assert bench.ncu_traffic()["dram_bytes_per_launch"] == 1.0
    with open(tmp_path / bench.PASS_SOURCES[0], "a") as f:
        f.write("\n// a comment changes nothing\n/* nor does\n   this one */\n")
    assert bench.ncu_traffic()["dram_bytes_per_launch"] == 1.0
    with open(tmp_path / bench.PASS_SOURCES[0], "a") as f:
        f.write("\nstatic const int changed_code = 1;\n")
    assert bench.ncu_traffic() is None
