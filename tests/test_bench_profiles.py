"""Host logic of bench.py (CPU): the reading of the committed ncu summaries (the
roofline's traffic comes from a summary only while its kernel source is unchanged
and, where the summary names them, for the same number of launches per step), and
the default line's serving block taken from a child process (its line kept even
when the child is ended in its cleanup; any failure recorded, never raised)."""
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


# --- the default line's serving block, from a child process (host logic) -------

LINE = ('{"metric": "serving p50/p99 ms (Poisson arrivals, continuous batching)", "failed": 0, '
        '"graph_launches": 0, "config": {"workload": "serving"}, "device_status": 0, '
        '"loads": [{"offered_qps": 1000.0, "qps": 950.0, "p50_ms": 60.0, "p99_ms": 130.0, "saturated": false, '
        '"mean_batch": 12.0, "per_db": {"a": {"p99_ms": 120.0}}}]}')


def child(code):
    return [sys.executable, "-c", code]


def test_serving_block_from_a_child_line():
    blk = bench.serving_block_from_child(child("print(%r)" % LINE), timeout_s=30)
    assert blk["p99_ms"] == 130.0 and blk["achieved_qps"] == 950.0 and blk["per_db_p99_ms"] == {"a": 120.0}
    assert "error" not in blk and "note" not in blk


def test_serving_block_keeps_the_line_of_a_child_stuck_in_cleanup():
    code = "import sys, time\nprint(%r, flush=True)\ntime.sleep(30)" % LINE
    blk = bench.serving_block_from_child(child(code), timeout_s=2)
    assert blk["p99_ms"] == 130.0 and "did not end" in blk["note"]


def test_serving_block_records_a_failed_or_silent_child():
    blk = bench.serving_block_from_child(child("import sys; sys.exit(3)"), timeout_s=30)
    assert blk["error"].startswith("RuntimeError: exit 3")
    blk = bench.serving_block_from_child(child("import sys\nprint(%r)\nsys.exit(1)" % LINE), timeout_s=30)
    assert blk["p99_ms"] == 130.0 and "exited with 1" in blk["note"]  # its line was printed first
    blk = bench.serving_block_from_child(child("import time; time.sleep(30)"), timeout_s=1)
    assert blk["error"].startswith("TimeoutExpired")
    blk = bench.serving_block_from_child(child("print('not json')"), timeout_s=30)
    assert "error" in blk
