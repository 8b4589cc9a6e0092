"""The bench line's `roofline.traffic` (host logic, no GPU): DRAM bytes per
launch from `profiles/traffic.json`, scaled by sites from a smaller capture
of the same kernel variant, and withheld (None) once the kernel source
differs from the one the counters were taken on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _entries():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)["k_step_tma1"]


def test_every_entry_names_its_report_and_its_capture():
    d = _entries()
    assert d
    for wl, e in d.items():
        assert os.path.exists(os.path.join(ROOT, "profiles", e["report"])), wl
        assert e["dram_bytes_per_launch"] > 0 and e["sites"] > 0 and e["steps_per_launch"] == 1
        if "scaled_from" in e:
            src = d[e["scaled_from"]]
            assert src["dram_bytes_per_launch"] == e["dram_bytes_per_launch"] and src["sites"] == e["sites"]
            assert "scaled_from" not in src          # scaled from a capture, not from another scaling


def test_traffic_is_scaled_by_sites_when_the_source_matches(monkeypatch):
    d = _entries()
    e = d["monolith_512"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: e["source_hash"])
    t = bench.measured_traffic("k_step_tma1", "monolith_512", 512 ** 3)
    assert abs(t - e["dram_bytes_per_launch"] * 512 ** 3 / e["sites"]) <= 1e-6 * t
    # bytes per site update of the capture carry over unchanged
    assert abs(t / 512 ** 3 - e["dram_bytes_per_launch"] / e["sites"]) < 1e-9


def test_traffic_is_withheld_after_a_kernel_change_or_without_a_capture(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.measured_traffic("k_step_tma1", "monolith_512", 512 ** 3) is None
    d = _entries()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: d["monolith_512"]["source_hash"])
    assert bench.measured_traffic("k_step_tma1", "no_such_workload", 1) is None
    assert bench.measured_traffic("no_such_kernel", "monolith_512", 1) is None


def test_the_source_hash_covers_the_step_kernels():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
