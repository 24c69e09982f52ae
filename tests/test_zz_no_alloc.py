"""lfd_superpixel_stats_noalloc, the entry point for callers that cannot
allocate device memory (stream capture, fixed memory plans, foreign
allocators), must give the superpixel statistics of the regular path
(lfd_set_input + lfd_get_superpixels) on two calls in a row: the second call
reuses the shared scratch array that the first one left filled.  Further
cases: every pixel format, a padded row pitch, an empty label and a label
outside the grid, the label limit, and a call recorded into a CUDA graph.

This file is collected last so that a run stopping at the first failure has
run every other test already."""
import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth

pytestmark = pytest.mark.gpu

FORMATS = {"rgba8": None, "rgba_f16": torch.float16, "rgba_bf16": torch.bfloat16, "rgba_f32": torch.float32}


def _views(lf, fmt):
    if fmt == "rgba8":
        return synth.quantize_rgba8(lf.rgb).cuda()
    return synth.to_rgba_float(lf.rgb, FORMATS[fmt]).cuda()


def _regular_stats(lfd, lf, views, labels, GW, GH, params):
    ctx = lfd.Context(0)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, GW, GH, params)
    ctx.synchronize()
    out = [ctx.get_superpixels(v)["stats"] for v in range(lf.rig.V)]
    ctx.close()
    return out


def _compare(got, ref):
    assert np.array_equal(got[:, 6], ref[:, 6])                            # pixel counts, exact
    ne = ref[:, 6] > 0
    assert np.allclose(got[ne, 0:2], ref[ne, 0:2], rtol=1e-6, atol=1e-5)   # centroids
    assert np.allclose(got[:, 2:5], ref[:, 2:5], rtol=1e-6, atol=1e-7)     # mean colours (0 when empty)
    assert np.allclose(got[:, 5], ref[:, 5], rtol=1e-5, atol=1e-6)         # minimum neighbour similarity


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def scene():
    lf = synth.make_config(1)
    lab0, GW, GH = synth.grid_labels(lf.rig.W, lf.rig.H, 16.0)
    lab2, _, _ = synth.grid_labels(lf.rig.W, lf.rig.H, 16.0, perturb=True, seed=11)
    lab1 = lab0.copy()
    lab1[lab1 == 23] = 24                  # label 23 is empty
    lf.labels = np.stack([lab0, lab1, lab2])
    return lf, GW, GH


def test_noalloc_superpixel_stats_match_the_regular_path_on_two_calls(lfd, scene):
    lf, GW, GH = scene
    views = _views(lf, "rgba8")
    labels = torch.from_numpy(np.ascontiguousarray(lf.labels)).cuda()
    params = synth.method_params(lf)
    ref = _regular_stats(lfd, lf, views, labels, GW, GH, params)
    S = GW * GH
    for v in (0, 2):                     # two calls in a row, different label maps
        out = torch.full((S, 8), float("nan"), dtype=torch.float32, device="cuda")
        lfd.superpixel_stats_noalloc(labels[v], views[v], GW, GH, params["alpha"], out)
        torch.cuda.synchronize()
        _compare(out.cpu().numpy(), ref[v])


@pytest.mark.parametrize("fmt", ["rgba_f16", "rgba_bf16", "rgba_f32"])
def test_noalloc_float_formats_and_an_empty_label(lfd, scene, fmt):
    lf, GW, GH = scene
    views = _views(lf, fmt)
    labels = torch.from_numpy(np.ascontiguousarray(lf.labels)).cuda()
    params = synth.method_params(lf)
    ref = _regular_stats(lfd, lf, views, labels, GW, GH, params)
    assert ref[1][23, 6] == 0                                # the emptied cell
    for v in range(lf.rig.V):
        out = torch.full((GW * GH, 8), float("nan"), dtype=torch.float32, device="cuda")
        lfd.superpixel_stats_noalloc(labels[v], views[v], GW, GH, params["alpha"], out)
        torch.cuda.synchronize()
        _compare(out.cpu().numpy(), ref[v])


def test_noalloc_padded_pitch(lfd, scene):
    """An FP16 view whose rows are 8 texels longer than the image: pitch =
    (W + 8) * 8 bytes."""
    lf, GW, GH = scene
    views = _views(lf, "rgba_f16")
    V, H, W, _ = views.shape
    padded = torch.full((V, H, W + 8, 4), float("nan"), dtype=torch.float16, device="cuda")
    padded[:, :, :W] = views
    labels = torch.from_numpy(np.ascontiguousarray(lf.labels)).cuda()
    params = synth.method_params(lf)
    ref = _regular_stats(lfd, lf, views, labels, GW, GH, params)
    for v in range(V):
        img = padded[v, :, :W]
        assert img.stride(0) == (W + 8) * 4
        out = torch.zeros((GW * GH, 8), dtype=torch.float32, device="cuda")
        lfd.superpixel_stats_noalloc(labels[v], img, GW, GH, params["alpha"], out)
        torch.cuda.synchronize()
        _compare(out.cpu().numpy(), ref[v])


def test_noalloc_ignores_labels_outside_the_grid(lfd, scene):
    """A pixel labelled >= grid_w * grid_h is left out of every statistic: the
    result equals the plain definition (count, mean position, mean colour of
    the remaining pixels of each label) written out in numpy."""
    lf, GW, GH = scene
    S = GW * GH
    views = _views(lf, "rgba8")
    lab = lf.labels[0].copy()
    lab[5, 7] = S + 3
    lab[100, 200] = 2 * S
    labels = torch.from_numpy(lab).cuda()
    out = torch.zeros((S, 8), dtype=torch.float32, device="cuda")
    lfd.superpixel_stats_noalloc(labels, views[0], GW, GH, 0.1, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    rgb = views[0, ..., :3].cpu().numpy().astype(np.float64) / 255.0
    yy, xx = np.mgrid[0:lab.shape[0], 0:lab.shape[1]]
    for s in range(S):
        m = lab == s
        n = int(m.sum())
        assert got[s, 6] == n
        if n:
            assert np.allclose(got[s, 0:2], [xx[m].mean(), yy[m].mean()], rtol=1e-6, atol=1e-5)
            assert np.allclose(got[s, 2:5], rgb[m].mean(axis=0), rtol=1e-6, atol=1e-7)
    assert got[:, 6].sum() == lab.size - 2


def test_noalloc_rejects_more_labels_than_its_scratch(lfd):
    from paper_1812_06856_gb300.lfd import LfdError
    H, W = 300, 300
    labels = torch.arange(H * W, dtype=torch.int32, device="cuda").reshape(H, W)
    img = torch.zeros((H, W, 4), dtype=torch.uint8, device="cuda")
    out = torch.zeros((H * W, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(LfdError) as e:
        lfd.superpixel_stats_noalloc(labels, img, W, H, 0.1, out)       # 90000 labels > 65536
    assert e.value.status == 1
    # at the limit itself the call runs
    lab2 = torch.arange(256 * 256, dtype=torch.int32, device="cuda").reshape(256, 256)
    img2 = torch.zeros((256, 256, 4), dtype=torch.uint8, device="cuda")
    out2 = torch.zeros((256 * 256, 8), dtype=torch.float32, device="cuda")
    lfd.superpixel_stats_noalloc(lab2, img2, 256, 256, 0.1, out2)
    torch.cuda.synchronize()
    assert torch.all(out2[:, 6] == 1)


def test_noalloc_call_recorded_into_a_cuda_graph(lfd, scene):
    """The reason the call exists: after one ordinary call (which looks up the
    scratch address), a second call is recorded by stream capture, where no
    allocation may happen, and the replayed graph gives the regular path's
    statistics."""
    lf, GW, GH = scene
    views = _views(lf, "rgba8")
    labels = torch.from_numpy(np.ascontiguousarray(lf.labels)).cuda()
    params = synth.method_params(lf)
    ref = _regular_stats(lfd, lf, views, labels, GW, GH, params)
    S = GW * GH
    warm = torch.zeros((S, 8), dtype=torch.float32, device="cuda")
    lfd.superpixel_stats_noalloc(labels[0], views[0], GW, GH, params["alpha"], warm)
    torch.cuda.synchronize()
    out = torch.full((S, 8), float("nan"), dtype=torch.float32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lfd.superpixel_stats_noalloc(labels[2], views[2], GW, GH, params["alpha"], out)
    g.replay()
    torch.cuda.synchronize()
    _compare(out.cpu().numpy(), ref[2])
