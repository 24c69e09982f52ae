"""Pins of the fusion oracle (Section III-D) against cases whose fused depth
follows from the definition by hand: agreeing candidates keep the closest
depth, a minority outlier loses to the majority, the agreement tolerance is
relative to the candidate, and a consistent surface seen by every view is
left unchanged."""
import numpy as np

from oracle import oracle as orc
from paper_1812_06856_gb300 import synth


def _cams(V, W, H, baseline=0.0):
    rig = synth.line_rig(V, baseline, 50.0, W, H) if baseline else synth.line_rig(V, 1e-9, 50.0, W, H)
    return rig.K, rig.R, rig.t


def _same_cams(V, W, H):
    K = np.stack([np.array([[50.0, 0.0, (W - 1) / 2], [0.0, 50.0, (H - 1) / 2], [0.0, 0.0, 1.0]])] * V)
    R = np.stack([np.eye(3)] * V)
    t = np.zeros((V, 3))
    return K, R, t


def test_identical_cameras_majority_and_closest_stable_depth():
    W, H = 7, 5
    K, R, t = _same_cams(3, W, H)
    # views see 1, 1, 5: the 5 disagrees with both others (stability -2); 1 keeps 0
    out, fl = orc.fuse(K, R, t, [np.full((H, W), 1.0), np.full((H, W), 1.0), np.full((H, W), 5.0)])
    assert all(np.all(o == 1.0) for o in out)
    # views see 1, 5, 5: 1 has stability -2, each 5 has +1 -1 = 0
    out, fl = orc.fuse(K, R, t, [np.full((H, W), 1.0), np.full((H, W), 5.0), np.full((H, W), 5.0)])
    assert all(np.all(o == 5.0) for o in out)
    # points land exactly on pixel centres: only the window edges (and their
    # neighbours) are within the margin of a decision
    assert all(not f[2:-2, 2:-2].any() for f in fl)


def test_agreement_tolerance_is_relative_to_the_candidate():
    W, H = 4, 3
    K, R, t = _same_cams(3, W, H)
    # 1.009 agrees with 1.0 (0.009 <= 0.01 * 1.0); 1.02 agrees with neither
    # stability(1.0) = +1 - 1 = 0 -> the closest stable candidate is 1.0
    out, _ = orc.fuse(K, R, t, [np.full((H, W), 1.0), np.full((H, W), 1.009), np.full((H, W), 1.02)], tau=0.01)
    assert all(np.all(o == 1.0) for o in out)
    # with tau = 0.03 everything agrees: the closest depth, 1.0, everywhere
    out, _ = orc.fuse(K, R, t, [np.full((H, W), 1.02), np.full((H, W), 1.009), np.full((H, W), 1.0)], tau=0.03)
    assert all(np.all(o == 1.0) for o in out)
    # with tau = 0.005 nothing agrees: every candidate has stability -2 -> 0
    out, _ = orc.fuse(K, R, t, [np.full((H, W), 1.02), np.full((H, W), 1.009), np.full((H, W), 1.0)], tau=0.005)
    assert all(np.all(o == 0.0) for o in out)


def test_no_depth_gives_no_depth_and_a_single_view_keeps_its_own():
    W, H = 5, 4
    K, R, t = _same_cams(2, W, H)
    out, _ = orc.fuse(K, R, t, [np.zeros((H, W)), np.zeros((H, W))])
    assert all(not o.any() for o in out)
    d = np.zeros((H, W))
    d[1, 2] = 3.0
    out, _ = orc.fuse(K, R, t, [d, np.zeros((H, W))])
    assert out[0][1, 2] == 3.0 and out[1][1, 2] == 3.0          # one candidate: stability 0


def test_fronto_parallel_plane_on_a_line_rig_is_a_fixed_point_and_outliers_are_replaced():
    """A plane at constant depth seen by parallel cameras projects between views
    with its depth unchanged: fusion leaves it as it is.  A patch of view 0
    pushed 30 % deeper is outvoted wherever the other two views see the plane."""
    W, H, z = 48, 32, 4.0
    rig = synth.line_rig(3, 0.1, 60.0, W, H)
    d = [np.full((H, W), z) for _ in range(3)]
    out, fl = orc.fuse(rig.K, rig.R, rig.t, d)
    for o in out:
        assert np.all(np.abs(o - z) <= 1e-12 * z)
    bad = [x.copy() for x in d]
    bad[0][8:20, 20:30] = 1.3 * z
    out, fl = orc.fuse(rig.K, rig.R, rig.t, bad)
    # interior of the patch: both other views land there (disparity 60*0.1/4 = 1.5 px, 3 px)
    assert np.all(np.abs(out[0][10:18, 22:28] - z) <= 1e-12 * z)
    # views 1 and 2 keep the plane: the displaced points of view 0 are one vote against two
    for o in out[1:]:
        assert np.all(np.abs(o[:, 4:W - 4] - z) <= 1e-12 * z)
