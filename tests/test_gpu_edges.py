"""Edge cases of the hot path against the FP64 oracle: the maximum label
count of the sweep, one superpixel per view (the whole image), uniform
images (every label ties up to the out-of-view samples), zero iterations, and
the largest iteration index of the propagation kernel (Eq. 4)."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth
import parity as PT
from test_gpu_parity import _iterate_compare, _sweep_compare, bind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


def _relabel(lf, labels, GW, GH):
    return dataclasses.replace(lf, labels=np.ascontiguousarray(labels, dtype=np.int32), GW=GW, GH=GH)


def test_sweep_at_the_maximum_label_count(lfd):
    lf = synth.make_config(1, scale=0.25)                 # 3 views 80x60, pitch 4
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=4096)     # LFD_MAX_LABELS: 16 label rounds per CTA
    o = PT.make_oracle(lf, rgb, params)
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print("\nsweep at 4096 labels:", rep)
    assert ok.all() and adm[ne].all() and rep["identical_when_decided"] == 1.0


def test_one_superpixel_per_view(lfd):
    """The whole image is one superpixel: the sweep walks it in many chunks,
    the propagation streams every pixel past the staged 320 and has no
    neighbour candidates and no triangles, so only the current plane is
    scored and kept."""
    base = synth.make_config(1, scale=0.5)                # 3 views 160x120
    lf = _relabel(base, np.zeros_like(base.labels), 1, 1)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=48, iterations=2)
    o = PT.make_oracle(lf, rgb, params)
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print("\none superpixel per view, sweep:", rep)
    assert ok.all() and adm[ne].all() and rep["identical_when_decided"] == 1.0
    ctx = bind(lfd, lf, views, labels, params)
    planes, _, _ = ctx.plane_sweep()
    state = planes.cpu().numpy()
    rep = {}
    out, same, adm = _iterate_compare(lfd, ctx, o, state, 1, np.arange(o.S_total, dtype=np.int32), rep)
    print("one superpixel per view, iteration 1:", rep)
    assert adm.all() and same.all()
    assert np.array_equal(out, state)                     # nothing to propagate, nothing to refine


def test_uniform_views_tie_to_the_lowest_label(lfd):
    """Uniform grey views: every in-view sample costs exactly 0, so a label's
    cost is T times its out-of-view samples and labels with equal counts tie
    exactly; both sides take the lowest k (Eq. 2 arg-min).  Only a projection
    within the oracle's margin of an image edge can change a count."""
    lf = synth.make_config(1, scale=0.5)
    lf = dataclasses.replace(lf, rgb=torch.full_like(lf.rgb, 0.5))
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=32, jitter=0)
    o = PT.make_oracle(lf, rgb, params)
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print("\nuniform views:", rep)
    assert ok.all() and adm[ne].all() and rep["identical_when_decided"] == 1.0


def test_zero_iterations_return_the_sweep(lfd):
    lf = synth.make_config(1, scale=0.5)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=32, iterations=0)
    ctx = bind(lfd, lf, views, labels, params)
    sweep, _, _ = ctx.plane_sweep()
    planes, depth = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    ctx.synchronize()
    assert torch.equal(planes, sweep)
    assert torch.isfinite(depth).all()


def test_largest_iteration_index(lfd):
    """Iteration index I = 64 (LFD_MAX_ITER_INDEX): the kernel of Eq. 4 has
    shrunk to the immediate neighbours; state-injected parity at I = 64."""
    lf = synth.make_config(1, scale=0.5)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=32, iterations=64)
    o = PT.make_oracle(lf, rgb, params)
    ctx = bind(lfd, lf, views, labels, params)
    planes, _, _ = ctx.plane_sweep()
    state = planes.cpu().numpy()
    rep = {}
    out, same, adm = _iterate_compare(lfd, ctx, o, state, 64, np.arange(o.S_total, dtype=np.int32), rep)
    print("\niteration index 64:", rep)
    assert adm.all() and rep["identical_when_decided"] == 1.0
    with pytest.raises(lfd.LfdError) as e:
        ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, dict(params, iterations=65))
    assert e.value.status == 1
