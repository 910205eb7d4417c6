"""The C ABI without a GPU: libxslam.so builds, loads, exports every call include/xslam.h declares,
and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re
import shutil

import numpy as np

import pytest

from paper_2405_02187_gb300 import xslam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(xslam_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(xslam.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("libxslam.so not built and no nvcc")
        from paper_2405_02187_gb300 import _build
        _build.build()
    return xslam.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 18
    bound = {name for name, _, _ in xslam.SYMBOLS}
    assert declared == bound, (declared ^ bound)
    for name in declared:
        assert hasattr(lib, name)


def test_pipeline_depth_matches_header():
    src = open(os.path.join(ROOT, "include", "xslam.h")).read()
    assert int(re.search(r"#define XSLAM_PIPELINE (\d+)", src).group(1)) == xslam.PIPELINE


def test_default_config(lib):
    c = xslam.default_config()
    assert c.icp_levels == 3 and list(c.icp_iters)[:3] == [10, 5, 4]
    assert abs(c.dist_gate_m - 0.1) < 1e-7 and abs(c.normal_gate_deg - 20) < 1e-6
    assert c.bilateral == 0 and c.w_max == 0


def _create(lib, dims=(8, 8, 8), voxel=0.01, trunc=0.04, intr=(100.0, 100.0, 31.5, 23.5, 64, 48), cfg=None,
            max_lanes=2):
    h = ctypes.c_void_p()
    K = xslam.Intrinsics(*intr)
    org = (ctypes.c_float * 3)(0, 0, 0)
    st = lib.xslam_create(ctypes.byref(h), *dims, voxel, trunc, org, ctypes.byref(K),
                          ctypes.byref(cfg) if cfg is not None else None, max_lanes, None)
    return st, h


@pytest.mark.parametrize("kw,msg", [
    (dict(dims=(1, 8, 8)), "dimensions"),
    (dict(voxel=0.0), "voxel"),
    (dict(trunc=-1.0), "truncation"),
    (dict(max_lanes=16), "max_lanes"),
    (dict(intr=(100.0, 100.0, 31.5, 23.5, 62, 48)), "divisible"),
    (dict(intr=(0.0, 100.0, 31.5, 23.5, 64, 48)), "focal"),
])
def test_create_rejects_bad_arguments(lib, kw, msg):
    st, h = _create(lib, **kw)
    assert st == xslam.EINVAL and not h.value
    assert msg in lib.xslam_last_error(None).decode()


def test_create_rejects_bad_config(lib):
    c = xslam.default_config()
    c.bilateral = 2
    st, _ = _create(lib, cfg=c)
    assert st == xslam.EINVAL and "bilateral" in lib.xslam_last_error(None).decode()
    c = xslam.default_config()
    c.icp_levels = 4
    st, _ = _create(lib, cfg=c)
    assert st == xslam.EINVAL
    c = xslam.default_config()
    c.depth_max_m = 0.1
    st, _ = _create(lib, cfg=c)
    assert st == xslam.EINVAL


def test_null_handle_calls(lib):
    assert lib.xslam_destroy(None) == xslam.OK
    assert lib.xslam_frame(None, None, 0, None, 0, None, None, None) == xslam.EINVAL
    assert lib.xslam_sync(None, None) == xslam.EINVAL
    assert lib.xslam_frame_submit(None, None, 0, None, 0, None) == xslam.EINVAL
    assert lib.xslam_frame_wait(None, 0, None, None, None) == xslam.EINVAL


@pytest.mark.parametrize("kw,msg", [
    (dict(dims=(1, 8, 8)), "dims"),
    (dict(voxel=0.0), "voxel"),
    (dict(max_runs=0), "max_runs"),
    (dict(max_runs=17), "max_runs"),
    (dict(intr=(0.0, 100.0, 31.5, 23.5, 64, 48)), "intrinsics"),
])
def test_plain_create_rejects_bad_arguments(lib, kw, msg):
    dims = kw.get("dims", (8, 8, 8))
    K = xslam.Intrinsics(*kw.get("intr", (100.0, 100.0, 31.5, 23.5, 64, 48)))
    org = (ctypes.c_float * 3)(0, 0, 0)
    h = ctypes.c_void_p()
    st = lib.xslam_plain_create(ctypes.byref(h), *dims, kw.get("voxel", 0.01), 0.04, org, ctypes.byref(K), None,
                                kw.get("max_runs", 2), None)
    assert st == xslam.EINVAL and not h.value
    assert msg in lib.xslam_plain_last_error(None).decode()


def test_plain_null_handle_calls(lib):
    assert lib.xslam_plain_destroy(None) == xslam.OK
    assert lib.xslam_plain_frame(None, None, 0, None, 0, None, None, None) == xslam.EINVAL
    assert lib.xslam_plain_set_pose(None, None) == xslam.EINVAL
    assert lib.xslam_plain_read_tsdf(None, 0, 0, None) == xslam.EINVAL


def test_icp_system_noalloc_binding_checks_sizes(lib):
    """The binding checks every buffer the C call reads before handing it over: a depth map of the
    wrong level size, a model with too few planes and a short pose block raise ValueError."""
    torch = pytest.importorskip("torch")
    from paper_2405_02187_gb300 import synth

    intr = synth.Intrinsics(100.0, 100.0, 31.5, 23.5, 64, 48)
    seeds = [(xslam.POSE0, 0, 1e-10), (xslam.DEPTH, -1, 1e-10)]
    L = 1 + len(seeds)
    T = np.zeros((L, 3, 4))
    good_d1 = torch.zeros(24 * 32)
    good_m = torch.zeros((1 + 6 * L) * 48 * 64)
    with pytest.raises(ValueError, match="depth"):
        xslam.icp_system_noalloc(torch.zeros(48 * 64), 1, intr, good_m, T, T, seeds, stream=0)
    with pytest.raises(ValueError, match="model"):
        xslam.icp_system_noalloc(good_d1, 1, intr, torch.zeros(6 * L * 48 * 64), T, T, seeds, stream=0)
    with pytest.raises(ValueError, match="doubles"):
        xslam.icp_system_noalloc(good_d1, 1, intr, good_m, T[:2], T, seeds, stream=0)
    with pytest.raises(ValueError, match="level"):
        xslam.icp_system_noalloc(good_d1, 3, intr, good_m, T, T, seeds, stream=0)
    # sizes right: the next check is the CUDA-tensor one, still before any library call
    with pytest.raises(TypeError, match="CUDA"):
        xslam.icp_system_noalloc(good_d1, 1, intr, good_m, T, T, seeds, stream=0)
