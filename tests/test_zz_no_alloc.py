"""lfd_superpixel_stats_noalloc, the entry point for callers that cannot
allocate device memory (stream capture, fixed memory plans, foreign
allocators), must give the superpixel statistics of the regular path
(lfd_set_input + lfd_get_superpixels) on two calls in a row: the second call
reuses the shared scratch array that the first one left filled.

This file is collected last so that a run stopping at the first failure has
run every other test already."""
import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_superpixel_stats_match_the_regular_path_on_two_calls():
    from paper_1812_06856_gb300 import lfd
    lfd.load()
    lf = synth.make_config(1)
    lab0, GW, GH = synth.grid_labels(lf.rig.W, lf.rig.H, 16.0)
    lab2, _, _ = synth.grid_labels(lf.rig.W, lf.rig.H, 16.0, perturb=True, seed=11)
    lf.labels = np.stack([lab0, lab0, lab2])
    views = synth.quantize_rgba8(lf.rgb).cuda()
    labels = torch.from_numpy(np.ascontiguousarray(lf.labels)).cuda()
    params = synth.method_params(lf)
    ctx = lfd.Context(0)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, GW, GH, params)
    ctx.synchronize()
    S = GW * GH
    for v in (0, 2):                     # two calls in a row, different label maps
        ref = ctx.get_superpixels(v)["stats"]
        out = torch.full((S, 8), float("nan"), dtype=torch.float32, device="cuda")
        lfd.superpixel_stats_noalloc(labels[v], views[v], GW, GH, params["alpha"], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got[:, 6], ref[:, 6])                       # pixel counts, exact
        ne = ref[:, 6] > 0
        assert np.allclose(got[ne, 0:2], ref[ne, 0:2], rtol=1e-6, atol=1e-5)   # centroids
        assert np.allclose(got[ne, 2:5], ref[ne, 2:5], rtol=1e-6, atol=1e-7)   # mean colours
        assert np.allclose(got[:, 5], ref[:, 5], rtol=1e-5, atol=1e-6)         # Eq. 11 minimum similarity
