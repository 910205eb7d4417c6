"""Host-side measurement logic of bench.py without a GPU: the algorithmic bytes per launch of each
frame stage against their closed forms at the 640x480, K = 6 workload, and the rule that an ncu traffic
record counts only while the kernel source it was taken on is unchanged."""
import hashlib
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _wl(width=640, height=480, iters=(10, 5, 4)):
    return types.SimpleNamespace(intr=types.SimpleNamespace(width=width, height=height), icp_iters=list(iters))


def test_icp_bytes_are_176_per_pixel_averaged_over_the_launches():
    # 4 B own depth + 4 B model depth + 24 B model vertex and normal on each of 7 lanes
    px = 10 * 640 * 480 + 5 * 320 * 240 + 4 * 160 * 120
    assert bench.algorithmic_bytes("icp", _wl(), 6, {}) == pytest.approx(px * 176 / 19, rel=1e-12)
    # one lane: 8 + 24 B per pixel
    assert bench.algorithmic_bytes("icp", _wl(iters=(1, 0, 0)), 0, {}) == 640 * 480 * 32


def test_fusion_bytes_are_64_per_updated_voxel_at_six_lanes():
    hw = 640 * 480
    assert bench.algorithmic_bytes("integrate", _wl(), 6, {"fused": 1e6}) == 64e6 + 4 * hw
    assert bench.algorithmic_bytes("integrate", _wl(), 0, {"fused": 1e6}) == 16e6 + 4 * hw


def test_raycast_bytes():
    hw = 640 * 480
    got = bench.algorithmic_bytes("raycast", _wl(), 6, {"fused": 2e6, "hits": 3e5})
    # outputs: depth + 6 floats on 7 lanes; F and W of the crossed voxels; 6 imaginary planes at 8 cells per hit
    assert got == hw * 4 * 43 + 2e6 * 8 + 3e5 * 8 * 8 * 4 * 6
    with pytest.raises(ValueError):
        bench.algorithmic_bytes("march", _wl(), 6, {})


def test_traffic_counts_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    src = tmp_path / "paper_2405_02187_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "fuse.cu").write_text("// kernel v1\n")
    (tmp_path / "profiles").mkdir()
    h1 = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    rec = {"room:integrate": {"src_sha256_16": h1, "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("integrate", "room") == 123
    assert bench.ncu_traffic("integrate", "other") is None
    (src / "fuse.cu").write_text("// kernel v2\n")
    assert bench.ncu_traffic("integrate", "room") is None
    (tmp_path / "profiles" / "traffic.json").unlink()
    assert bench.ncu_traffic("integrate", "room") is None


def test_committed_traffic_records_name_their_kernel_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for key, e in d.items():
        if key.startswith("_"):
            continue
        stage = key.split(":")[1]
        assert stage in bench.KERNEL_SRC
        assert len(e["src_sha256_16"]) == 16 and e["dram_bytes_per_launch"] > 0
