"""bench.py's reading of the committed ncu summaries (host logic, CPU): the
roofline's traffic comes from a summary only while its kernel source is unchanged
and, where the summary names them, for the same number of launches per step."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def write_summary(tmp_path, monkeypatch, source_text, lines):
    src = tmp_path / "kernel.cu"
    src.write_text(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    body = "\n".join(["# header", "kernel: k", "workload: w", "batch: 4"] + lines +
                     ["source_sha256: " + bench.sha256_of(str(src)), "traffic_bytes_per_launch: 1234"])
    (prof / "k_w_b4.txt").write_text(body + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return str(src)


def test_traffic_read_while_source_unchanged(tmp_path, monkeypatch):
    src = write_summary(tmp_path, monkeypatch, "kernel v1", [])
    assert bench.profile_traffic("k", "w", 4, src) == 1234.0
    assert bench.profile_traffic("k", "w", 4, src, launches_per_step=3.0) == 1234.0  # no count named: no check
    assert bench.profile_traffic("k", "w", 8, src) is None                          # no summary for batch 8
    open(src, "w").write("kernel v2")
    assert bench.profile_traffic("k", "w", 4, src) is None                          # source changed since


def test_traffic_only_for_the_same_launches_per_step(tmp_path, monkeypatch):
    src = write_summary(tmp_path, monkeypatch, "kernel", ["launches_per_step: 4"])
    assert bench.profile_traffic("k", "w", 4, src, launches_per_step=4.0) == 1234.0
    assert bench.profile_traffic("k", "w", 4, src, launches_per_step=2.0) is None   # other K-chunks
    assert bench.profile_traffic("k", "w", 4, src) == 1234.0


def test_traffic_per_launch_count(tmp_path, monkeypatch):
    src = write_summary(tmp_path, monkeypatch, "kernel",
                        ["launches_per_step: 4", "traffic_bytes_per_launch@2: 5000", "traffic_bytes_per_launch@4: 1234"])
    assert bench.profile_traffic("k", "w", 4, src, launches_per_step=2.0) == 5000.0
    assert bench.profile_traffic("k", "w", 4, src, launches_per_step=4.0) == 1234.0
    assert bench.profile_traffic("k", "w", 4, src, launches_per_step=1.0) is None
