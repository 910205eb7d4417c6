"""Host-side measurement logic of bench.py without a GPU: the algorithmic bytes per launch of each
frame stage against their closed forms at the 640x480, K = 6 workload, the ray cast's distinct voxel
reads against a brute-force count, the rule that an ncu traffic record counts only while the kernel
source it was taken on is unchanged, and the line's handling of a failing companion section."""
import hashlib
import json
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _wl(width=640, height=480, iters=(10, 5, 4)):
    return types.SimpleNamespace(intr=types.SimpleNamespace(width=width, height=height), icp_iters=list(iters))


def test_icp_bytes_are_192_per_pixel_iteration():
    # the scope table's figure: 24 B own vertex and normal + 24 B model vertex and normal on each of 7 lanes
    px = 10 * 640 * 480 + 5 * 320 * 240 + 4 * 160 * 120
    assert bench.icp_bytes_per_frame(_wl(), 6) == px * 192
    # one cooperative launch per frame carries all of it; 19 launches share it
    assert bench.algorithmic_bytes("icp", _wl(), 6, {}) == px * 192
    assert bench.algorithmic_bytes("icp", _wl(), 6, {}, launches_per_frame=19) == pytest.approx(px * 192 / 19)
    # one lane: 24 + 24 B per pixel
    assert bench.algorithmic_bytes("icp", _wl(iters=(1, 0, 0)), 0, {}) == 640 * 480 * 48


def test_fusion_bytes_are_64_per_updated_voxel_at_six_lanes():
    hw = 640 * 480
    assert bench.algorithmic_bytes("integrate", _wl(), 6, {"fused": 1e6}) == 64e6 + 4 * hw
    assert bench.algorithmic_bytes("integrate", _wl(), 0, {"fused": 1e6}) == 16e6 + 4 * hw


def test_raycast_bytes():
    hw = 640 * 480
    got = bench.algorithmic_bytes("raycast", _wl(), 6, {"march_voxels": 2e6, "refine_voxels": 3e5})
    # outputs: depth + 6 floats on 7 lanes; Re F of the marched voxels; all 7 lanes of the refined ones
    assert got == hw * 4 * 43 + 2e6 * 4 + 3e5 * 4 * 7
    with pytest.raises(ValueError):
        bench.algorithmic_bytes("march", _wl(), 6, {})


def _brute_voxel_reads(intr, T, hit, dims, voxel, origin, step, m0, m1):
    """The same sets by explicit per-ray loops over every sample alpha_m with m0 <= m <= m1."""
    nx, ny, nz = dims
    R, t = np.asarray(T)[:, :3], np.asarray(T)[:, 3]
    march, refine = set(), set()

    def cell(g):
        if all(0 <= g[i] < dims[i] - 1 for i in range(3)):
            i, j, k = (int(np.floor(c)) for c in g)
            return {(i + a) + nx * ((j + b) + ny * (k + c)) for a in (0, 1) for b in (0, 1) for c in (0, 1)}
        return set()

    for v in range(intr.height):
        for u in range(intr.width):
            d = R @ np.array([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, 1.0])
            gp = lambda a: (t + a * d - np.asarray(origin)) / voxel - 0.5  # noqa: E731
            h = float(hit[v, u])
            ins = [m for m in range(m0, m1 + 1) if cell(gp(m * step))]
            if not ins:
                continue
            end = int(np.floor(h / step)) + 1 if h > 0 else ins[-1]
            for m in range(ins[0], end + 1):
                march |= cell(gp(m * step))
            if h > 0:
                mh = int(np.floor(h / step))
                pts = [gp(mh * step), gp((mh + 1) * step)]
                vt = gp(h)
                for i in range(3):
                    for sgn in (1.0, -1.0):
                        q = vt.copy()
                        q[i] += sgn
                        pts.append(q)
                for q in pts:
                    refine |= cell(q)
    return len(march), len(refine)


def test_raycast_voxel_reads_match_brute_force():
    torch = pytest.importorskip("torch")
    from paper_2405_02187_gb300 import synth
    intr = synth.Intrinsics(6.0, 6.0, 3.5, 2.5, 8, 6)
    dims, voxel, origin, step = (12, 10, 14), 0.05, (-0.3, -0.25, 0.05), 0.05
    c, s_ = np.cos(0.2), np.sin(0.2)
    T = np.array([[c, 0.0, s_, 0.01], [0.0, 1.0, 0.0, -0.02], [-s_, 0.0, c, 0.0]])
    rng = np.random.default_rng(0)
    hit = rng.uniform(0.2, 0.6, (6, 8))
    hit[rng.random((6, 8)) < 0.3] = 0.0
    m0, m1 = 2, 20
    got = bench.raycast_voxel_reads(intr, T, torch.tensor(hit), dims, voxel, origin, step, m0, m1, chunk=7)
    assert got == _brute_voxel_reads(intr, T, hit, dims, voxel, origin, step, m0, m1)
    assert got[0] > 100 and got[1] > 20


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


def test_a_failing_companion_section_leaves_the_headline():
    # a companion section (batched, second order, learned proposal) that raises is reported in the line
    # as an error object; the line's summaries pass it through instead of failing on its missing keys
    def boom(*_):
        raise RuntimeError("no memory")

    r = bench.run_section("batched", boom, None, None, 0)
    assert r == {"error": "batched: RuntimeError: no memory"}
    assert bench._batched_summary(r) == r
    assert bench._second_summary({"error": "e"}) == {"error": "e"}
    assert bench._learned_summary({"error": "e"}) == {"error": "e"}
    assert bench._batched_summary(None) is None and bench._learned_summary(None) is None
    assert bench.run_section("batched", lambda *a: {"value": 1.0}) == {"value": 1.0}
