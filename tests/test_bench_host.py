"""Host logic of bench.py that needs no GPU: the clock sampler, and the
lookup of the committed traffic capture (end of file).

A stand-in `nvidia-smi` on PATH prints the queried fields every 50 ms (first
clocks at 2070 MHz with no throttle reason, then 1500 MHz with sw_power_cap
active); the sampler must keep only the samples taken inside the window it is
given, take their median SM clock and report the active reasons.
"""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FAKE = """#!/bin/sh
n=0
while true; do
  if [ $n -lt 10 ]; then
    echo "2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
  else
    echo "1500, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
  fi
  n=$((n + 1))
  sleep 0.05
done
"""


def _with_fake(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))


def test_sampler_keeps_window_and_reports_reasons(tmp_path, monkeypatch):
    _with_fake(tmp_path, monkeypatch)
    import bench
    c = bench.ClockSampler(0)
    c.start()
    assert c.lines, "sampler returned before its first sample"
    t0 = time.perf_counter()
    time.sleep(0.2)             # samples of the first phase (2070 MHz, 0.5 s long)
    t1 = time.perf_counter()
    time.sleep(0.6)             # later samples (1500 MHz, power cap) fall outside [t0, t1]
    early = c.stop(t0, t1)
    assert early["sm_mhz"] == 2070.0 and early["reasons"] == [], early
    assert early["samples"] >= 1


def test_sampler_sees_power_cap(tmp_path, monkeypatch):
    _with_fake(tmp_path, monkeypatch)
    import bench
    c = bench.ClockSampler(0)
    c.start()
    time.sleep(0.8)
    t0 = time.perf_counter()
    time.sleep(0.3)
    t1 = time.perf_counter()
    late = c.stop(t0, t1)
    assert late["sm_mhz"] == 1500.0, late
    assert late["sm_max_mhz"] == 2070.0
    assert late["reasons"] == ["sw_power_cap"]


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    import bench
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_record_keyed_to_its_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed capture only while the files
    of the captured kernel's translation unit are those it was taken on: an
    edit to another source keeps it, an edit to a listed file voids it."""
    import json
    import shutil
    import bench
    from paper_1401_6750_gb300 import build
    files = ["eo.cu", "dslash.cuh", "common.cuh", "tsm.h"]
    here = build.source_digest(files)
    csrc, inc = tmp_path / "csrc", tmp_path / "include"
    shutil.copytree(build.CSRC, csrc)
    shutil.copytree(build.INCLUDE, inc)
    monkeypatch.setattr(build, "CSRC", str(csrc))
    monkeypatch.setattr(build, "INCLUDE", str(inc))
    assert build.source_digest(files) == here  # another checkout of the same files
    rec = {"kernel_class": "k", "dram_bytes_per_launch": 1234, "source_files": files,
           "source_digest": build.source_digest(files)}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "roofline_traffic.txt").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "__file__", str(tmp_path / "bench.py"))
    assert bench.measured_traffic("k") == 1234
    assert bench.measured_traffic("other") is None
    with open(csrc / "contract.cu", "a") as fh:  # not part of the kernel's unit
        fh.write("\n// edit\n")
    assert bench.measured_traffic("k") == 1234
    with open(csrc / "dslash.cuh", "a") as fh:
        fh.write("\n// edit\n")
    assert bench.measured_traffic("k") is None
