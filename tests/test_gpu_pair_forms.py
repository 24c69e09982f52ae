"""Homography specialisations (lfd_set_pair_forms / lfd_pair_form).

The library classifies the camera pairs of a bound input as general, affine
(P row 3 = (0, 0, P22), q_z = 0) or translation (affine and P's 2 x 2 block =
P22 I) and runs specialised sweep and propagation kernels.  Checked here:
  * the classification of the three rigs (line and grid of parallel cameras
    with equal intrinsics: translation; arc: general);
  * the affine form gives the general form's sweep costs and propagation
    planes bit for bit (same arithmetic, value for value);
  * the translation form's sweep costs differ from the general form's only
    by the rounding of the sample position (the general form rounds absolute
    FP32 positions, the translation form splits each label's shift into
    integer and fraction in FP64): within the parity tolerance (relative
    1e-4 plus the TSSD floor); its labels are the general form's wherever
    the two best costs are apart by more than that, and its propagation
    (which runs the affine form) is bit-identical;
  * each form against the FP64 oracle (the parity protocol of the sweep).
"""
import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth
import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


def _bound(lfd, lf, views, labels, params, max_form):
    ctx = lfd.Context(0)
    ctx.set_pair_forms(max_form)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    return ctx


def test_rig_classification(lfd):
    for cfg, scale, fmt, expect in ((1, 1.0, "rgba8", 2), (3, 0.125, "rgba_f16", 2), (2, 0.25, "rgba8", 0)):
        lf = synth.make_config(cfg, scale=scale)
        views, labels, _ = PT.gpu_inputs(lf, fmt)
        params = synth.method_params(lf, num_labels=32)
        for cap in (0, 1, 2):
            ctx = _bound(lfd, lf, views, labels, params, cap)
            assert ctx.pair_form() == min(expect, cap), (cfg, cap)
            ctx.close()
    ctx = lfd.Context(0)
    with pytest.raises(lfd.LfdError):
        ctx.set_pair_forms(3)
    with pytest.raises(lfd.LfdError):
        ctx.pair_form()                       # nothing bound yet
    ctx.close()


@pytest.mark.parametrize("cfg,scale,fmt", [(1, 1.0, "rgba8"), (3, 0.125, "rgba_f16"), (3, 0.125, "rgba_bf16")])
def test_forms_agree(lfd, cfg, scale, fmt):
    lf = synth.make_config(cfg, scale=scale)
    views, labels, rgb = PT.gpu_inputs(lf, fmt)
    params = synth.method_params(lf, num_labels=64)
    res = {}
    for form in (0, 1, 2):
        ctx = _bound(lfd, lf, views, labels, params, form)
        assert ctx.pair_form() == form
        planes, lab, costs = ctx.plane_sweep(want_labels=True, want_costs=True)
        ctx.synchronize()
        state = planes.clone()
        out, choice, energy = ctx.iterate(1, state, want_choice=True)
        ctx.synchronize()
        res[form] = dict(lab=lab.cpu().numpy(), costs=costs.cpu().numpy().astype(np.float64),
                         planes=planes.cpu(), out=out.cpu(), state=state)
        ctx.close()
    # affine = general, bit for bit
    assert np.array_equal(res[1]["costs"], res[0]["costs"])
    assert np.array_equal(res[1]["lab"], res[0]["lab"])
    assert torch.equal(res[1]["out"], res[0]["out"])
    # translation: both forms inside the oracle's intervals (which span the
    # window-edge decisions that position rounding can move), and within the
    # parity tolerance of each other wherever the oracle flagged nothing
    o = PT.make_oracle(lf, rgb, params)
    sw = o.sweep(np.arange(o.S_total), want_costs=True)
    c0, c2 = res[0]["costs"], res[2]["costs"]
    present = res[0]["lab"] >= 0
    floor = PT.tssd_abs_floor(o)[:, None] + PT.ABS
    for c in (c0, c2):
        assert PT.within(c[present], sw["cost_lo"][present], sw["cost_hi"][present], absf=floor[present]).all()
    tol = PT.REL * np.abs(c0) + floor
    unfl = (sw["cost_lo"] == sw["cost_hi"]) & present[:, None]
    assert np.all(np.abs(c2[unfl] - c0[unfl]) <= tol[unfl])
    # labels: identical unless the general form's best two costs are within the tolerance
    srt = np.sort(c0[present], axis=1)
    gap = srt[:, 1] - srt[:, 0]
    clear = gap > 2 * tol[present].max(axis=1)
    assert np.array_equal(res[2]["lab"][present][clear], res[0]["lab"][present][clear])
    print(f"\nconfig {cfg} {fmt}: translation vs general: max rel cost diff "
          f"{float(np.max(np.abs(c2[present] - c0[present]) / np.maximum(np.abs(c0[present]), 1e-12))):.3g}, "
          f"labels identical {float(np.mean(res[2]['lab'][present] == res[0]['lab'][present])):.4f} "
          f"({int((~clear).sum())} of {int(present.sum())} superpixels with a near-tie)")
    # the propagation runs the affine form under both: from the same state, the same planes
    ctx = _bound(lfd, lf, views, labels, params, 2)
    out2, _, _ = ctx.iterate(1, res[0]["state"].cuda(), want_choice=True)
    ctx.synchronize()
    assert torch.equal(out2.cpu(), res[0]["out"])
    ctx.close()


@pytest.mark.parametrize("form", [0, 2])
def test_form_against_oracle(lfd, form):
    """Sweep parity of the general and translation forms on the 3-view line rig."""
    lf = synth.make_config(1, scale=0.5)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=48)
    o = PT.make_oracle(lf, rgb, params)
    ctx = _bound(lfd, lf, views, labels, params, form)
    planes, lab, costs = ctx.plane_sweep(want_labels=True, want_costs=True)
    ctx.synchronize()
    lab, costs = lab.cpu().numpy(), costs.cpu().numpy().astype(np.float64)
    sw = o.sweep(np.arange(o.S_total), want_costs=True)
    ne = sw["label"] >= 0
    floor = PT.tssd_abs_floor(o)[:, None] + PT.ABS
    assert PT.within(costs[ne], sw["cost_lo"][ne], sw["cost_hi"][ne], absf=floor[ne]).all()
    same = lab == sw["label"]
    adm = np.array([same[i] or PT.admissible(-sw["cost_lo"][i, lab[i]], -sw["cost_hi"][i]) for i in range(len(lab))])
    assert adm[ne].all()
    ctx.close()
