"""Host-side pieces of bench.py: the algorithmic bytes behind the roofline, the replica
aggregation, and the source hashes that decide whether a committed DRAM-traffic capture
still describes the kernel."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_pass_bytes_is_one_read_and_one_write_of_six_fields():
    # six real fields of 512^3 FP32 in and six packed half spectra out: 12 x 512^3 / 2 complex x 8 B
    assert bench.pass_bytes("z_fused", 512, 4) == 6 * 512 ** 3 * 4 * 2 == 6442450944
    assert bench.pass_bytes("x_r2c", 64, 8) == 2 * bench.pass_bytes("x_r2c", 64, 4)


def test_replica_value_counts_every_rank():
    assert bench.whole_job_value(1, 1e9, 1000.0) == 1e9
    assert bench.whole_job_value(4, 1e9, 2000.0) == 2e9


def test_source_hash_tracks_the_kernel_sources():
    h = bench.source_sha("z_fused")
    assert h == bench.source_sha("z_fused") and len(h) == 16
    assert h != bench.source_sha("y_fft")
    for kind, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(ROOT, "paper_2210_06232_gb300", "csrc", f)), (kind, f)


def test_traffic_entry_is_ignored_when_sources_differ(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    good = {"bytes_per_launch": 123.0, "source_sha": bench.source_sha("z_fused")}
    stale = {"bytes_per_launch": 456.0, "source_sha": "0" * 16}
    (prof / "traffic.json").write_text(json.dumps({"z_fused_fp32_512": good, "y_fft_fp32_512": stale}))
    (tmp_path / "paper_2210_06232_gb300").mkdir()
    os.symlink(os.path.join(ROOT, "paper_2210_06232_gb300", "csrc"), tmp_path / "paper_2210_06232_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("z_fused_fp32_512") == 123.0
    assert bench.traffic_for("y_fft_fp32_512") is None
    assert bench.traffic_for("x_r2c_fp32_512") is None
