"""Host side of the serving workload: the moving rigs and the frame walk."""
import numpy as np

from paper_1812_06856_gb300 import synth


def test_serving_rig_moves_one_step_per_frame():
    r = synth.make_serving_rig("B", "cpu", keyframes=3, scale=0.05)
    assert r.V == 9 and len(r.views) == 3 and r.views[0].shape[-1] == 4
    seq = [r.keyframe_of(f) for f in range(10)]
    assert seq == [0, 1, 2, 1, 0, 1, 2, 1, 0, 1]
    for a, b in zip(seq, seq[1:]):
        d = r.rigs[b].centres() - r.rigs[a].centres()
        assert np.allclose(np.linalg.norm(d, axis=1), r.step)       # <= 2 cm per frame
        assert np.allclose(d[:, 1:], 0.0)
    assert r.labels.shape == (9, r.rigs[0].H, r.rigs[0].W)
    assert int(r.labels.max()) == r.GW * r.GH - 1
