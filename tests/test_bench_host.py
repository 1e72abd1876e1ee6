"""Host-side pieces of bench.py that need no GPU.

The JSON line's `roofline.traffic` is read from the committed ncu summary of
the warp-tile kernel, and only while the kernel source is the one the
counters were taken on: any edit of the source must turn it into null rather
than report counters of another kernel.  The workload names that key those
records must stay the ones the bench prints.  The clock record of the timed
region (median SM clock, throttle reasons) is parsed from nvidia-smi's CSV,
here fed by a stand-in process.
"""

import os
import re
import shutil

import bench

WORKLOADS = ("json", "clike", "arith", "clike_block", "clike_block_framed")
PROFILE = os.path.join("profiles", "lex_warps_dram_512mib.md")
SOURCE = os.path.join("paper_2608_03473_gb300", "csrc", "lexwarp.cu")


def _tree(tmp_path, src_text=None):
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / "paper_2608_03473_gb300" / "csrc")
    shutil.copy(os.path.join(bench.ROOT, PROFILE), tmp_path / PROFILE)
    if src_text is None:
        shutil.copy(os.path.join(bench.ROOT, SOURCE), tmp_path / SOURCE)
    else:
        (tmp_path / SOURCE).write_text(src_text)


def test_traffic_records_cover_the_default_workload():
    text = open(os.path.join(bench.ROOT, PROFILE)).read()
    keys = {k for k, _, _ in re.findall(r"<!-- traffic (\S+) (\d+) ([0-9a-f]{64}) -->", text)}
    assert bench.workload_name("json", 512) in keys
    assert keys <= {bench.workload_name(w, 512) for w in WORKLOADS}


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    text = open(os.path.join(bench.ROOT, PROFILE)).read()
    recs = re.findall(r"<!-- traffic (\S+) (\d+) ([0-9a-f]{64}) -->", text)
    key, val, sha = recs[0]
    src = open(os.path.join(bench.ROOT, SOURCE), "rb").read()
    import hashlib
    same = hashlib.sha256(src).hexdigest() == sha

    a = tmp_path / "same"
    _tree(a)
    monkeypatch.setattr(bench, "ROOT", str(a))
    assert bench.profiled_traffic(key) == (int(val) if same else None)
    assert bench.profiled_traffic("no_such_workload") is None

    b = tmp_path / "edited"
    _tree(b, src.decode() + "\n// edited\n")
    monkeypatch.setattr(bench, "ROOT", str(b))
    assert bench.profiled_traffic(key) is None


def test_workload_and_metric_names_are_distinct():
    names = [bench.workload_name(w, 512) for w in WORKLOADS]
    metrics = [bench.metric_name(w, 512) for w in WORKLOADS]
    assert len(set(names)) == len(names) and len(set(metrics)) == len(metrics)
    assert all(w in bench.CUTS for w in WORKLOADS)


class _FakeSmi:
    """Stands in for `nvidia-smi --query-gpu=... -lms`: canned CSV rows."""

    def __init__(self, rows):
        self.rows = rows

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return "\n".join(self.rows) + "\n", ""


def test_clock_sampler_reads_median_clock_and_throttle_reasons(monkeypatch):
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbled line"]
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeSmi(rows))
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]

    rows2 = ["0, 1410, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active"]
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeSmi(rows2))
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["sm_mhz"] == 1410 and c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    def missing(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
