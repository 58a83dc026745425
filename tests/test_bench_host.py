"""Host logic of bench.py (no GPU): the DRAM traffic it reports for the dominant kernel comes from the
committed ncu summary only while the kernel's sources are the ones that capture was taken with."""
import json

import bench


def test_source_digest_is_stable_and_covers_the_class_files():
    assert bench.kernel_source_hash("spread") == bench.kernel_source_hash("spread")
    assert bench.kernel_source_hash("fft_x") == bench.kernel_source_hash("fft_y")     # the same file
    assert bench.kernel_source_hash("spread") != bench.kernel_source_hash("fft_x")
    assert bench.kernel_source_hash("interp") != bench.kernel_source_hash("prep")


def test_traffic_is_reported_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"kernel": "k", "dram_bytes": 12345, "source_hash": bench.kernel_source_hash("spread")}
    (prof / "traffic.json").write_text(json.dumps({"per_launch": {"w_mixed": {"spread": entry}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the temporary root holds no sources: stand in for the digest of the unchanged ones
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: entry["source_hash"] if k == "spread" else "x")
    assert bench.ncu_traffic("spread", "w_mixed") == 12345
    assert bench.ncu_traffic("spread", "other_workload") is None
    assert bench.ncu_traffic("fft_x", "w_mixed") is None
    # a source edit after the capture: the figure is dropped, not reported
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "changed")
    assert bench.ncu_traffic("spread", "w_mixed") is None


def test_committed_traffic_entries_have_positive_byte_counts():
    with open(f"{bench.ROOT}/profiles/traffic.json") as f:
        d = json.load(f)
    for workload, classes in d["per_launch"].items():
        for cls, e in classes.items():
            assert cls in bench.KERNEL_FILES, (workload, cls)
            assert isinstance(e["dram_bytes"], int) and e["dram_bytes"] > 0
            assert len(e["source_hash"]) == 16
