"""Host-side pieces of bench.py that need no GPU.

The JSON line's `roofline.traffic` is read from the committed ncu summary of
the warp-tile kernel, and only while the kernel source is the one the
counters were taken on: any edit of the source must turn it into null rather
than report counters of another kernel.  The workload names that key those
records must stay the ones the bench prints.
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
