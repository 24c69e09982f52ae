"""GPU SLIC (lfd_slic) against the FP64 SLIC oracle, the segmentation step the
method runs before Section III-A.

State-injected steps compare exactly: the seeds (Lab within FP32 rounding, xy
identical), one assignment from the same centres (labels identical wherever the
oracle's two smallest distances are not within its margin), one update from
the GPU's own labels (means within FP32 summation error).  The free-running
segmentation (seeds + 10 iterations) is compared by label agreement, since a
near-tie that goes the other way moves a mean and the runs drift apart.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1812_06856_gb300 import synth
import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


def blobs(H, W, seed):
    """Piecewise-smooth colour image: random discs over a gradient, with noise."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.stack([x / W, y / H, 0.5 + 0.3 * np.sin(x / 7.0)], axis=-1)
    for _ in range(12):
        cx, cy, r = rng.uniform(0, W), rng.uniform(0, H), rng.uniform(4, max(6, min(W, H) / 3))
        img[(x - cx) ** 2 + (y - cy) ** 2 < r * r] = rng.uniform(0, 1, 3)
    img += rng.normal(0, 0.02, img.shape)
    return np.clip(img, 0, 1)


def device_views(rgb, fmt):
    """(V, H, W, 4) device tensor of format fmt and the float64 RGB it holds."""
    t = torch.from_numpy(np.ascontiguousarray(rgb))
    if fmt == "rgba8":
        q = synth.quantize_rgba8(t)
        return q.cuda(), synth.rgba8_as_float(q).numpy()
    dt = {"rgba_f16": torch.float16, "rgba_bf16": torch.bfloat16, "rgba_f32": torch.float32}[fmt]
    v = synth.to_rgba_float(t, dt)
    return v.cuda(), v[..., :3].to(torch.float64).numpy()


CASES = [  # (H, W, GW, GH, fmt)
    (96, 128, 16, 12, "rgba8"),
    (67, 101, 9, 7, "rgba_f16"),          # ragged cells
    (50, 70, 1, 1, "rgba_f32"),           # one cell
    (17, 23, 23, 17, "rgba8"),            # one pixel per cell
    (200, 300, 37, 23, "rgba_bf16"),
]


@pytest.mark.parametrize("H,W,GW,GH,fmt", CASES)
def test_slic_steps_state_injected(lfd, H, W, GW, GH, fmt):
    m = 10.0
    views, rgb = device_views(np.stack([blobs(H, W, 1), blobs(H, W, 2)]), fmt)
    ctx = lfd.Context(0)
    # seeds
    lab0, seeds = ctx.slic(views, GW, GH, m, iterations=0, want_centres=True)
    ctx.synchronize()
    seeds = seeds.cpu().numpy().astype(np.float64)
    for v in range(2):
        ref = orc.slic_seeds(rgb[v], GW, GH)
        assert np.array_equal(seeds[v][:, 3:], ref[:, 3:])
        assert np.allclose(seeds[v][:, :3], ref[:, :3], rtol=1e-5, atol=2e-4)
    # one assignment from the same (FP32) centres
    c0 = torch.from_numpy(seeds.astype(np.float32))
    c0[..., 0] += 3.0 * torch.sin(torch.arange(GW * GH, dtype=torch.float32))    # move them off the grid
    c0[..., 3] += 0.3 * torch.cos(torch.arange(GW * GH, dtype=torch.float32))
    labA = ctx.slic(views, GW, GH, m, iterations=0, centres_in=c0.cuda())
    ctx.synchronize()
    labA = labA.cpu().numpy()
    flagged = 0.0
    for v in range(2):
        ref, fl = orc.slic_assign(rgb[v], GW, GH, c0[v].numpy().astype(np.float64), m)
        ok = fl == 0
        assert np.array_equal(labA[v][ok], ref[ok]), f"view {v}: {np.sum(labA[v][ok] != ref[ok])} labels differ"
        assert np.all((labA[v] >= 0) & (labA[v] < GW * GH))
        flagged = max(flagged, float(fl.mean()))
    assert flagged < 0.01
    # one update: the means of the first assignment's pixels
    _, c1 = ctx.slic(views, GW, GH, m, iterations=1, centres_in=c0.cuda(), want_centres=True)
    ctx.synchronize()
    c1 = c1.cpu().numpy().astype(np.float64)
    for v in range(2):
        ref = orc.slic_update(rgb[v], GW, GH, labA[v], c0[v].numpy().astype(np.float64))
        assert np.allclose(c1[v], ref, rtol=2e-5, atol=2e-3)
    print(f"\nSLIC {W}x{H} grid {GW}x{GH} {fmt}: flagged share {flagged:.2e}")
    ctx.close()


def test_slic_free_running_agrees_with_oracle(lfd):
    lf = synth.make_config(1)
    views, _, rgb = PT.gpu_inputs(lf, "rgba8")
    rgb = rgb.numpy() if hasattr(rgb, "numpy") else rgb
    GW, GH = lf.GW, lf.GH
    ctx = lfd.Context(0)
    lab, cen = ctx.slic(views, GW, GH, 10.0, iterations=10, want_centres=True)
    ctx.synchronize()
    lab, cen = lab.cpu().numpy(), cen.cpu().numpy()
    rates = []
    for v in range(min(4, lab.shape[0])):
        ref, cref = orc.slic(rgb[v], GW, GH, 10.0, 10)
        rates.append(float(np.mean(lab[v] == ref)))
        assert np.all((lab[v] >= 0) & (lab[v] < GW * GH))
    print(f"\nSLIC free-running ({lf.name}, {GW}x{GH} cells): label agreement {rates}")
    assert min(rates) >= 0.97
    ctx.close()


def test_slic_labels_drive_the_estimate(lfd):
    """SLIC label maps go into the estimate unchanged (any label map in range
    is accepted) and give finite depths close to the grid segmentation's."""
    lf = synth.make_config(1, device="cuda")
    params = synth.method_params(lf)
    views, labels, _ = PT.gpu_inputs(lf, "rgba8")
    ctx = lfd.Context(0)
    sl = ctx.slic(views, lf.GW, lf.GH, 10.0, iterations=10)
    pg, dg = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params, want_depth=True)
    ps, ds = ctx.estimate(views, sl, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params, want_depth=True)
    ctx.synchronize()
    ds, dg = ds.cpu().numpy(), dg.cpu().numpy()
    assert np.all(np.isfinite(ds))
    both = (ds > 0) & (dg > 0)
    assert both.mean() > 0.9
    rel = np.abs(ds[both] - dg[both]) / dg[both]
    print(f"\nSLIC vs grid superpixels: median relative depth difference {np.median(rel):.3g}")
    assert np.median(rel) < 0.05
    ctx.close()
