"""The benchmark's byte model (the roofline's algorithmic bytes) and its
bookkeeping, checked by hand on a tiny tensor: per mode m,
  B(m) = nnz * (4 (N-1) + 4) + sum_{n != m} U_n R s_f + I_m R 4
with U_n the distinct rows of mode n that some nonzero touches."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_bytes_model_by_hand():
    # dims 4 x 3 x 5; nonzeros touch rows {0, 2} of mode 0, {1} of mode 1, {0, 3, 4} of mode 2
    idx = np.array([[0, 1, 0], [2, 1, 3], [0, 1, 4], [2, 1, 0]], dtype=np.int32)
    c = synth.Coo((4, 3, 5), idx, np.ones(4, np.float32))
    U = bench.distinct_rows(c)
    assert U == [2, 1, 3]
    R = 8
    # stream: 4 nonzeros x (2 coordinates + 1 value) x 4 B = 48 B
    # mode 0: inputs U1 + U2 = 4 rows x 8 x 4 B = 128; output 4 rows x 8 x 4 B = 128 -> 304
    # mode 1: inputs 2 + 3 = 5 rows -> 160; output 3 rows -> 96 -> 304
    # mode 2: inputs 2 + 1 = 3 rows -> 96; output 5 rows -> 160 -> 304
    assert bench.bytes_model(c, R, 4, U) == [304, 304, 304]
    # 16-bit factors halve only the gathered rows: 48 + 64 + 128, 48 + 80 + 96, 48 + 48 + 160
    assert bench.bytes_model(c, R, 2, U) == [240, 224, 256]


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while the MTTKRP sources
    hash to the captured version."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "same")
    (prof / "mttkrp_toy_traffic.txt").write_text("kernel_source_sha: same\ndram_bytes_per_launch_f32: 1234\n")
    assert bench.recorded_traffic("toy") == 1234.0
    (prof / "mttkrp_toy_traffic.txt").write_text("kernel_source_sha: other\ndram_bytes_per_launch_f32: 1234\n")
    assert bench.recorded_traffic("toy") is None
    assert bench.recorded_traffic("missing") is None


def test_workload_config_names_the_workload():
    class A:
        segment_items = 0
        inner_order = "lexicographic"
        short_rows = 0
        stream_memory = "device"
    w = synth.WORKLOADS["zipf3"]
    cfg = bench.workload_config(w, A())
    assert cfg["workload"] == "zipf3" and cfg["nnz"] == 200_000_000 and cfg["rank"] == 32
    assert "model" not in cfg and cfg["l2"].startswith("inputs_exceed_l2")
