"""Host logic of bench.py (no GPU): the convolution byte count of the packed
m = 0 transforms and the traffic figure that is reported only while the kernel
and table sources still have the hashes the capture was taken with."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_convolution_bytes_per_point():
    import bench
    # lmax 4, 10 bins: 100 complex arrays at 56 B and 25 packed pairs of real m = 0 arrays at 72 B
    assert bench.conv_bytes_per_point(4, 10) == 100 * 56 + 25 * 72 == 7400
    # an odd bin count leaves one unpacked m = 0 array per l
    assert bench.conv_bytes_per_point(0, 3) == 72 + 56
    assert bench.conv_bytes_per_point(1, 2) == 2 * 56 + 2 * 72


def test_profiled_traffic_follows_the_source_hashes(tmp_path, monkeypatch):
    import bench
    t = bench.profiled_traffic(256)
    assert t is not None and t > 0
    assert abs(bench.profiled_traffic(128) * 8 - t) < 1e-6 * t  # scaled by grid points
    # a copy of the tree whose kernel source differs reports no traffic
    for rel in ("profiles/tc4_kernel_traffic.txt", "paper_2210_10206_gb300/csrc/sbg_api.cu",
                "paper_2210_10206_gb300/csrc/sbg_tc.cu"):
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), tmp_path / rel)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic(256) == t
    with open(tmp_path / "paper_2210_10206_gb300/csrc/sbg_tc.cu", "a") as f:
        f.write("\n")
    assert bench.profiled_traffic(256) is None
