"""Host logic of the benchmark that needs no GPU: roofline.traffic comes from the committed
ncu summary of the dominant kernel, scaled by coordinates, and only while the kernel sources
still hash to the version that was captured."""
import os
import shutil

import bench


def test_traffic_scales_with_coordinates():
    t1 = bench.profiled_traffic("lambda_sweep_kernel", 1_000_000)
    t2 = bench.profiled_traffic("lambda_sweep_kernel", 2_000_000)
    assert t1 is not None and t1 > 0
    assert abs(t2 - 2 * t1) <= 1e-9 * t2
    # the committed capture: between 10 and 200 KB of DRAM traffic per coordinate
    assert 10e3 < t1 / 1e6 < 200e3


def test_traffic_is_null_for_other_kernels_and_changed_sources(tmp_path, monkeypatch):
    assert bench.profiled_traffic("theta_sweep_kernel", 1000) is None  # no capture committed
    # a copy of the tree whose kernel source differs by one byte: the capture no longer applies
    root = tmp_path / "tree"
    for rel in bench.SWEEP_SOURCES + ["profiles/lambda_sweep_kernel-q5000-bounded.md"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic("lambda_sweep_kernel", 1000) is not None
    src = root / bench.SWEEP_SOURCES[0]
    src.write_bytes(src.read_bytes() + b" ")
    assert bench.profiled_traffic("lambda_sweep_kernel", 1000) is None
