"""Host logic of bench.py that needs no GPU: the clock / throttle record taken
during the timed region, read from a stand-in for nvidia-smi."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/sh
printf '0, 2070, 2070, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active\\n'
printf '0, 2055, 2070, 1012.4, 0x4, Not Active, Not Active, Not Active, Active\\n'
printf '0, 2070, 2070, 1020.0, 0x0, Not Active, Not Active, Not Active, Not Active\\n'
printf '0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active\\n'
printf 'garbage line\\n'
exec sleep 30
"""


def test_clock_sampler_parses_a_record(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text(FAKE)
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    rec = s.stop()
    assert rec is not None
    assert rec["samples"] == 4  # the malformed line is skipped
    assert rec["sm_mhz"] == 2070.0  # median of 2070, 2055, 2070 (N/A skipped)
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() is None
