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
    import hashlib
    import bench
    # a tree whose capture file carries the hashes of its current sources
    srcs = ("paper_2210_10206_gb300/csrc/sbg_api.cu", "paper_2210_10206_gb300/csrc/sbg_tc.cu")
    for rel in srcs:
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), tmp_path / rel)
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    with open(tmp_path / "profiles/tc4_kernel_traffic.txt", "w") as f:
        f.write("# test capture\n")
        for rel in srcs:
            f.write(f"sha256 {rel} {hashlib.sha256(open(tmp_path / rel, 'rb').read()).hexdigest()}\n")
        f.write("grid 128\ndram_bytes_read 5000000000\ndram_bytes_write 4000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t = bench.profiled_traffic(256)
    assert t == (5000000000 + 4000000) * 8  # scaled by grid points
    assert abs(bench.profiled_traffic(128) * 8 - t) < 1e-6 * t
    # once the kernel source differs the figure is no longer reported
    with open(tmp_path / "paper_2210_10206_gb300/csrc/sbg_tc.cu", "a") as f:
        f.write("\n")
    assert bench.profiled_traffic(256) is None


def test_algorithmic_flops_of_the_roofline_are_counted_from_the_definition():
    # the roofline's numerator: the (Lambda, M) terms of the 4PCF sum of Eq. mu
    # with m3 >= 0 (even Lambda at lmax 4, every M, as Algorithm 6 loops them)
    # times the bin triples b1 <= b2 <= b3, 4 flops per term and grid point
    import itertools

    import bench
    from oracle import sarabande_oracle as O
    terms = 0
    for l1, l2, l3 in O.lambda_list(bench.LMAX4):
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -(m1 + m2)
                if 0 <= m3 <= l3:
                    terms += 1
    triples = sum(1 for _ in itertools.combinations_with_replacement(range(bench.NB), 3))
    assert (terms, triples) == (bench.ALG_TERMS_LM, bench.ALG_BIN_TRIPLES) == (490, 220)
    assert abs(terms * triples * 256 ** 3 * 4 - 7.2343e12) < 1e9
