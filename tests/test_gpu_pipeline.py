"""The pipelined frame calls (xslam_frame_submit / xslam_frame_wait) against xslam_frame: the same
frames in the same order give the same poses and derivatives bit for bit, whether the depth maps come
from numpy, pinned host tensors or the device, with up to XSLAM_PIPELINE frames in flight, mixed with
synchronous frames; each ticket reports its own frame's tracking failure; the queue and ticket rules."""
import numpy as np
import pytest

from gpu_helpers import gpu_seeds, make_handle
from oracle import pipeline as P
from paper_2405_02187_gb300 import synth, xslam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEEDS = [P.Seed(P.POSE0, 0), P.Seed(P.TRUNC), P.Seed(P.DEPTH, -1)]
EMPTY = 6  # this frame's depth map is all zeros: ICP fails on it and the frame is fused at the previous pose


@pytest.fixture(scope="module")
def orbit():
    return synth.small_orbit(frames=12)


def _inputs(wl):
    """Frame k's depth map as a numpy array, a pinned host tensor or a device tensor, in turn."""
    out = []
    for k in range(len(wl.depth)):
        d = np.ascontiguousarray(wl.depth[k] if k != EMPTY else np.zeros_like(wl.depth[k]), np.float32)
        if k % 3 == 0:
            out.append(d)
        elif k % 3 == 1:
            out.append(torch.from_numpy(d.copy()).pin_memory())
        else:
            out.append(torch.tensor(d, device="cuda"))
    return out


def _reference(wl, ins, sd):
    x = make_handle(wl, max_lanes=len(sd))
    x.set_pose(wl.poses[0])
    ref = [x.frame(d, sd) for d in ins]
    x.close()
    return ref


def _same(r, g, k):
    assert r[3] == g[3], k
    for u, v in zip(r[:3], g[:3]):
        assert np.array_equal(u, v), k


def test_pipelined_frames_equal_synchronous(orbit):
    sd = gpu_seeds(SEEDS)
    ins = _inputs(orbit)
    ref = _reference(orbit, ins, sd)
    assert ref[EMPTY][3] == xslam.ENOTRACK
    assert all(r[3] == xslam.OK for k, r in enumerate(ref) if k != EMPTY)
    x = make_handle(orbit, max_lanes=len(sd))
    x.set_pose(orbit.poses[0])
    got, tickets = [], []
    for d in ins:
        tickets.append(x.submit(d, sd))
        if len(tickets) - len(got) == xslam.PIPELINE:  # keep the queue full
            got.append(x.wait(tickets[len(got)]))
    while len(got) < len(tickets):
        got.append(x.wait(tickets[len(got)]))
    x.close()
    assert tickets == list(range(len(ins)))
    for k, (r, g) in enumerate(zip(ref, got)):
        _same(r, g, k)


def test_pipelined_and_synchronous_frames_mix(orbit):
    sd = gpu_seeds(SEEDS[:2])
    ins = _inputs(orbit)
    ref = _reference(orbit, ins, sd)
    x = make_handle(orbit, max_lanes=len(sd))
    x.set_pose(orbit.poses[0])
    got = {}
    pending = []
    for k, d in enumerate(ins):
        if k % 4 == 3:  # a synchronous frame with earlier frames still outstanding
            got[k] = x.frame(d, sd)
            for j, t in pending:
                got[j] = x.wait(t)
            pending = []
        else:
            pending.append((k, x.submit(d, sd)))
    for j, t in pending:
        got[j] = x.wait(t)
    x.close()
    for k, r in enumerate(ref):
        _same(r, got[k], k)


def test_pipeline_queue_and_ticket_rules(orbit):
    sd = gpu_seeds(SEEDS[:1])
    x = make_handle(orbit, max_lanes=1)
    x.set_pose(orbit.poses[0])
    t = [x.submit(orbit.depth[k], sd) for k in range(xslam.PIPELINE)]
    with pytest.raises(xslam.XSlamError) as e:
        x.submit(orbit.depth[xslam.PIPELINE], sd)  # the queue is full
    assert e.value.status == xslam.ESTATE
    with pytest.raises(xslam.XSlamError) as e:
        x.wait(t[1])  # not the oldest outstanding ticket
    assert e.value.status == xslam.EINVAL
    with pytest.raises(xslam.XSlamError) as e:
        x.submit(orbit.depth[0], gpu_seeds([P.Seed(P.POSE0, 1)]))  # seeds cannot change mid-sequence
    assert e.value.status == xslam.ESTATE
    for tk in t:
        assert x.wait(tk)[3] == xslam.OK
    with pytest.raises(xslam.XSlamError) as e:
        x.wait(t[-1])  # already delivered
    assert e.value.status == xslam.EINVAL
    # a reset finishes and drops the outstanding frames; the next sequence numbers on
    t2 = x.submit(orbit.depth[0], sd)
    x.reset()
    with pytest.raises(xslam.XSlamError) as e:
        x.wait(t2)
    assert e.value.status == xslam.EINVAL
    x.set_pose(orbit.poses[0])
    t3 = x.submit(orbit.depth[0], sd)
    assert t3 == t2 + 1
    pose, _, _, st = x.wait(t3)
    assert st == xslam.OK and np.allclose(pose, orbit.poses[0][:3], atol=1e-12)
    x.close()


def test_pipelined_headline_frames_equal_synchronous():
    """640x480 room in 256^3 with the bilateral filter, K = 6 POSE0 lanes, pinned host depth: the
    configuration the end-to-end throughput is measured on."""
    wl = synth.room_walk(seed=2, frames=8, device="cpu", resident=False)
    sd = [(P.POSE0, j, 1e-10) for j in range(6)]
    host = torch.from_numpy(np.ascontiguousarray(wl.depth, np.float32)).pin_memory()
    ins = [host[k] for k in range(len(wl.depth))]
    ref = _reference(wl, ins, sd)
    x = make_handle(wl, max_lanes=6)
    x.set_pose(wl.poses[0])
    got = []
    t_prev = None
    for d in ins:  # the bench's pattern: submit frame k, then read frame k - 1
        t = x.submit(d, sd)
        if t_prev is not None:
            got.append(x.wait(t_prev))
        t_prev = t
    got.append(x.wait(t_prev))
    x.close()
    for k, (r, g) in enumerate(zip(ref, got)):
        assert r[3] == xslam.OK
        _same(r, g, k)
