"""CPU checks of bench.py's bookkeeping that needs no GPU: the source regions
the symmetric step kernel's DRAM-traffic figure is tied to, and how a stale
figure is dropped."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_09712_gb300", "csrc")


def test_hash_regions_exist():
    # the hash covers named regions; a renamed marker must fail here, not in
    # the benchmark
    hdr = open(os.path.join(CSRC, "cts_internal.h")).read()
    ker = open(os.path.join(CSRC, "cts_kernels.cu")).read()
    assert hdr.count("// ---- kernel launchers") == 1
    assert ker.count("// Update alone:") == 1
    assert ker.count("const VariantEntry kVariants[]") == 1
    assert ker.index("const VariantEntry kVariants[]") < ker.index("#undef CTS_V")
    # both step kernels lie inside the hashed part
    assert ker.index("step_kernel(StepArgs a") < ker.index("// Update alone:")
    assert ker.index("sym_kernel(StepArgs a") < ker.index("// Update alone:")


def test_hash_is_deterministic_and_hex():
    h = bench.kernel_source_hash()
    assert h == bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_traffic_is_dropped_when_the_source_hash_differs(monkeypatch):
    path = os.path.join(ROOT, "profiles", "sym_kernel_traffic.json")
    d = json.load(open(path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: d["kernel_source_hash"])
    assert bench.profiled_traffic() == d["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic() is None


def test_committed_traffic_summary_is_consistent():
    d = json.load(open(os.path.join(ROOT, "profiles", "sym_kernel_traffic.json")))
    total = d["dram_read_bytes_captured"] + d["dram_write_bytes_captured"]
    assert d["dram_bytes_per_launch_captured"] == total
    # scaled from the captured events to the benchmark's 64-event launch
    assert d["dram_bytes_per_launch"] == total * 64 / d["events_in_capture"]
