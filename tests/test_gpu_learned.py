"""What the trained proposal network gains over the method without it (constant-velocity ICP).

The network is trained on the GPU (include/xslam_mlp.h) on frame pairs of room walks that the
X-KinectFusion step itself tracked, then judged on walks it has not seen: its guess of the camera
motion must lie closer to the true motion than the constant-velocity guess, and ICP seeded with it
(accepted only where its converged coarse-level residual is no worse) must track at least as well
as constant-velocity ICP."""
import numpy as np
import pytest

from paper_2405_02187_gb300 import learn, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    ds = learn.make_dataset(n_traj=40, frames=16, reverse=True, seed=40000)
    m, losses, _ = learn.train(ds, epochs=20, mirror=True)
    yield m, ds.scale, losses
    m.close()


def test_training_converges(trained):
    _, _, losses = trained
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.6 * losses[0]


def test_network_start_is_closer_than_constant_velocity(trained):
    m, scale, _ = trained
    wl = synth.room_walk(seed=41000, frames=80, stride=2, device="cuda", resident=True)
    e = learn.start_errors(m, scale, wl)
    print({k: round(float(v.mean()), 3) for k, v in e.items()})
    assert e["network"].mean() < 0.8 * e["constant_velocity"].mean()


def _run(wl, seed_mode, mlp, scale):
    r = learn.track(wl, learn.handle_config(wl, seed_mode, 1e-5), [], mlp=mlp, scale=scale, judge_level=2,
                    timed=False)
    dt, _ = learn.pose_errors(r["poses"], wl.poses)
    return r["failures"], float(dt.mean()), r["counters"]


def test_second_start_tracks_no_worse(trained):
    """A fast camera with inertia and abrupt changes every 10 frames: ICP from one start (constant
    velocity, or the previous pose) against the same start plus the network's, judged."""
    m, scale, _ = trained
    wl = synth.room_smooth(seed=42000, frames=60, dims=256, voxel=0.01, step_m=0.04, step_deg=3.0, jerk_every=10,
                           device="cuda")
    res = {}
    for seed_mode, name in ((1, "cv"), (0, "prev")):
        res[name] = _run(wl, seed_mode, None, scale)
        res[name + "+proposal"] = _run(wl, seed_mode, m, scale)
    print(res)
    for name in ("cv", "prev"):
        f0, e0, _ = res[name]
        f1, e1, cnt = res[name + "+proposal"]
        assert cnt["judged"] == len(wl.poses) - 1 and 0 < cnt["accepted"] <= cnt["judged"]
        assert f1 <= f0
        assert e1 <= e0 + 0.005
