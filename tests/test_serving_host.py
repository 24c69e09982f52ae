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


def test_fast_grid_labels_equal_reference():
    for (W, H, p, pert, seed) in [(64, 48, 8, True, 3), (97, 61, 11, True, 5), (80, 60, 16, False, 0),
                                  (130, 70, 9.5, True, 11)]:
        a, gw, gh = synth.grid_labels(W, H, p, pert, seed=seed)
        b, gw2, gh2 = synth.grid_labels_fast(W, H, p, pert, seed=seed)
        assert (gw, gh) == (gw2, gh2)
        assert np.array_equal(a, b.numpy())


def test_mix_workload_shapes():
    mix = synth.make_mix(3, "cpu", scale=0.1)
    assert len(mix) == 3
    for m in mix:
        V = m.rig.V
        assert 4 <= V <= 16 and m.views.shape[0] == V and m.labels.shape[0] == V
        assert 128 <= m.params["num_labels"] <= 256 and m.params["iterations"] == 6
        assert int(m.labels.max()) < m.GW * m.GH
    assert len({m.params["lf_index"] for m in mix}) == 3
