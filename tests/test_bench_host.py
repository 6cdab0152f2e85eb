"""Host logic of bench.py that needs no GPU: the DRAM-traffic record that the
roofline object quotes is well formed, and a figure is reported only while
the kernel's source still has the hash recorded with it."""
import hashlib
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_is_well_formed():
    kernels = set()
    for line in open(os.path.join(ROOT, "profiles", "dram_traffic.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        assert len(f) >= 5, line
        assert int(f[1]) > 0
        assert os.path.exists(os.path.join(ROOT, f[2])), f[2]
        assert re.fullmatch(r"[0-9a-f]{64}", f[3]), f[3]
        kernels.add(f[0])
    assert {"k_deposit_lp", "k_project_lp"} <= kernels  # the two roofline objects


def test_traffic_reported_only_for_the_recorded_source(tmp_path, monkeypatch):
    import bench

    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# header\n"
        f"k_a 1234 k.cu {sha} workload\n"
        f"k_b 5678 k.cu {'0' * 64} workload\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k_a") == 1234
    assert bench.profiled_traffic("k_b") is None   # source changed since the capture
    assert bench.profiled_traffic("k_c") is None   # never captured
    src.write_text("kernel source, edited\n")
    assert bench.profiled_traffic("k_a") is None
