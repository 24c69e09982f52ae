"""Batched frames (Section III-E across light fields): several light fields in
one pass of the sweep and propagation kernels give the same bits as separate
calls; every launch shape, the autotuner and CUDA-graph replay give the same
bits as the default launch."""
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


def _item(lf, views, labels, params):
    return dict(views=views, labels=labels, K=lf.rig.K, R=lf.rig.R, t=lf.rig.t, GW=lf.GW, GH=lf.GH, params=params)


@pytest.fixture(scope="module")
def two_rigs():
    """A 3-view line rig (64 labels, 4 iterations) and an 8-view arc rig at
    quarter resolution (256 labels, 6 iterations, its own jitter key)."""
    a = synth.make_config(1)
    b = synth.make_config(2, scale=0.25)
    va, la, _ = PT.gpu_inputs(a, "rgba8")
    vb, lb, _ = PT.gpu_inputs(b, "rgba8")
    pa = synth.method_params(a)
    pb = synth.method_params(b, lf_index=1)
    return [(a, va, la, pa), (b, vb, lb, pb)]


def _separate(lfd, rigs):
    out = []
    for lf, v, l, p in rigs:
        ctx = lfd.Context(0)
        planes, depth = ctx.estimate(v, l, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, p)
        ctx.synchronize()
        out.append((planes.clone(), depth.clone()))
    return out


def _split(rigs, planes):
    res, base = [], 0
    for lf, v, l, p in rigs:
        n = lf.rig.V * lf.GW * lf.GH
        res.append(planes[base:base + n])
        base += n
    return res


def test_batch_equals_separate_calls(lfd, two_rigs):
    ref = _separate(lfd, two_rigs)
    ctx = lfd.Context(0)
    planes, depths = ctx.estimate_batch([_item(*r) for r in two_rigs])
    ctx.synchronize()
    for (rp, rd), bp, bd in zip(ref, _split(two_rigs, planes), depths):
        assert torch.equal(rp, bp)
        assert torch.equal(rd, bd)
    # the staged calls see the batch with global view numbering; neighbour
    # views stay inside each light field
    va = two_rigs[0][0].rig.V
    for v in range(ctx.V):
        nb = ctx.get_superpixels(v)["neighbours"]
        nb = nb[nb >= 0]
        inside = (nb < va) if v < va else (nb >= va)
        assert inside.all() and len(nb) > 0


@pytest.mark.parametrize("opt", [
    dict(sweep_threads=128),
    dict(sweep_persistent=0),
    dict(prop_blocks=7),
    dict(prop_persistent=0),
    dict(sweep_threads=128, sweep_persistent=1, prop_blocks=7, prop_persistent=1),
    dict(prop_batch=16),
    dict(order_bands=1),
    dict(prop_batch=16, order_bands=1, prop_persistent=0),
    dict(prop_coop=1),
    dict(prop_coop=1, prop_batch=16, prop_blocks=7),
    dict(prop_coop=1, prop_batch=16, order_bands=1),
])
def test_launch_shapes_give_identical_bits(lfd, two_rigs, opt):
    ctx = lfd.Context(0)
    p0, d0 = ctx.estimate_batch([_item(*r) for r in two_rigs])
    ctx.synchronize()
    p0, d0 = p0.clone(), [d.clone() for d in d0]
    ctx2 = lfd.Context(0)
    p1, d1 = ctx2.estimate_batch([_item(*r) for r in two_rigs], options=opt)
    ctx2.synchronize()
    cfg = ctx2.launch_config()
    for k, v in opt.items():
        assert cfg[k] == v
    assert torch.equal(p0, p1)
    assert all(torch.equal(a, b) for a, b in zip(d0, d1))


def test_autotune_picks_a_valid_shape_and_same_bits(lfd, two_rigs):
    ctx = lfd.Context(0)
    p0, d0 = ctx.estimate_batch([_item(*r) for r in two_rigs])
    ctx.synchronize()
    p0 = p0.clone()
    ctx2 = lfd.Context(0)
    p1, _ = ctx2.estimate_batch([_item(*r) for r in two_rigs], options=dict(autotune=1))
    ctx2.synchronize()
    cfg = ctx2.launch_config()
    assert cfg["sweep_threads"] in (128, 256) and cfg["prop_blocks"] in (7, 8)
    assert cfg["sweep_persistent"] in (0, 1) and cfg["prop_persistent"] in (0, 1)
    assert cfg["prop_batch"] in (16, 32) and cfg["order_bands"] in (1, 16) and cfg["prop_coop"] in (0, 1)
    assert torch.equal(p0, p1)
    # counters count the frame only, not the timing runs
    h, s = ctx2.counters()
    h0, s0 = ctx.counters()
    assert (h, s) == (h0, s0)


def test_graph_replay_reads_new_frame_contents(lfd, two_rigs):
    stream = torch.cuda.Stream()
    items = [_item(*r) for r in two_rigs]
    ctx = lfd.Context(0)
    ctx.profile_enable(False)
    with torch.cuda.stream(stream):
        out = ctx.estimate_batch(items, options=dict(graph=1), stream=stream)
    stream.synchronize()
    planes, depths = out
    first = planes.clone()
    launches_first = [n for _, n in ctx.profile_read().values()]
    # next frame: new image contents in the same buffers
    a, va, la, pa = two_rigs[0]
    saved = va.clone()
    g = torch.Generator(device="cpu").manual_seed(7)
    noise = torch.randint(-6, 7, va.shape, generator=g, dtype=torch.int16).to(va.device)
    va.copy_((saved.to(torch.int16) + noise).clamp(0, 255).to(torch.uint8))
    stream.wait_stream(torch.cuda.current_stream())
    try:
        with torch.cuda.stream(stream):
            ctx.estimate_batch(items, options=dict(graph=1), out=out, stream=stream)
        stream.synchronize()
        launches_replay = [n for _, n in ctx.profile_read().values()]
        assert launches_replay == launches_first and sum(launches_replay) > 0
        ref = _separate(lfd, two_rigs)
        for (rp, rd), bp, bd in zip(ref, _split(two_rigs, planes), depths):
            assert torch.equal(rp, bp)
            assert torch.equal(rd, bd)
        assert not torch.equal(first, planes)      # the replay did read the new images
    finally:
        va.copy_(saved)


def test_batch_rejects_mixed_formats_and_graph_on_default_stream(lfd, two_rigs):
    a, va, la, pa = two_rigs[0]
    b, vb, lb, pb = two_rigs[1]
    vb16 = synth.to_rgba_float(b.rgb, torch.float16).to(vb.device)
    ctx = lfd.Context(0)
    with pytest.raises(lfd.LfdError, match="pixel format"):
        ctx.estimate_batch([_item(a, va, la, pa), _item(b, vb16, lb, pb)])
    with pytest.raises(lfd.LfdError, match="non-default stream"):
        ctx.estimate_batch([_item(a, va, la, pa)], options=dict(graph=1),
                           stream=torch.cuda.default_stream())
    with pytest.raises(lfd.LfdError, match="batch options"):
        ctx.estimate_batch([_item(a, va, la, pa)], options=dict(sweep_threads=64))
    with pytest.raises(lfd.LfdError, match="batch options"):
        ctx.estimate_batch([_item(a, va, la, pa)], options=dict(prop_batch=24))
