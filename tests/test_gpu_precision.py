"""Reduced-precision input forms against the FP64 oracle on the FP64 rendering.

The parity tests give the oracle exactly the colours the GPU sees; here the
oracle sees the unrounded FP64 rendering instead, so the statistics measure
what storing the views as RGBA8, FP16, BF16 or FP32 costs.  Per configuration
and format, on a deterministic sample of superpixels: sweep labels identical
to the FP64 arg-min, median relative error of the label costs and the share
inside the oracle's interval (which spans a window edge or rounding boundary
the FP64 evaluation finds within its margin) widened by 1e-4, and for the first
refinement iteration (state-injected from the GPU's own sweep) the chosen
plane identical to the FP64 choice and the depth within 0.5 %.  Config 1 also
runs free (sweep + all iterations) on both sides: the flip rate is the share
of superpixels whose final plane differs.
"""
import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth
import parity as PT

pytestmark = pytest.mark.gpu

CASES = [
    (1, ("rgba8", "rgba_f16", "rgba_bf16", "rgba_f32")),
    (2, ("rgba8", "rgba_f16", "rgba_bf16", "rgba_f32")),
    (3, ("rgba_f16", "rgba_bf16", "rgba_f32")),
]
# Bounds on the sampled statistics: the observed figures (printed) less a
# stated margin.  Labels: at most one near-tie in 32 sampled superpixels may
# go the other way (observed 31/32 on configs 2 and 3 for every format,
# FP32 included, and 96/96 on config 1); iteration-1 depths within 0.5 %:
# at most one in 96 (observed all); free-running config 1 depths within
# 0.5 %: >= 99 % (observed 99.3-99.9 %).  Median relative cost error per
# storage format (observed: RGBA8 1.0-1.8e-4, BF16 0.6-1.4e-4, FP16
# 1.2-1.8e-5, FP32 0.07-1.1e-5) and the share of costs inside the FP64
# interval widened by 1e-4 for the formats whose rounding is below it
# (observed FP32 >= 0.998, FP16 >= 0.976).
LABEL_FLOOR = 0.95
DEPTH_FLOOR = 0.985
FREE_DEPTH_FLOOR = 0.99
COST_MEDIAN_MAX = {"rgba8": 3e-4, "rgba_bf16": 2.5e-4, "rgba_f16": 4e-5, "rgba_f32": 3e-5}
COST_INSIDE_MIN = {"rgba_f16": 0.95, "rgba_f32": 0.99}


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


@pytest.mark.parametrize("cfg,fmts", CASES)
def test_input_precision_against_fp64(lfd, cfg, fmts):
    lf = synth.make_config(cfg, device="cuda")
    params = synth.method_params(lf)
    rgb64 = lf.rgb.detach().cpu().to(torch.float64)
    o = PT.make_oracle(lf, rgb64, params)
    rng = np.random.default_rng(100 + cfg)
    n_items = 32 if cfg > 1 else 96
    items = np.sort(rng.choice(o.S_total, size=n_items, replace=False)).astype(np.int32)
    sw = o.sweep(items, want_costs=True)
    present = sw["label"] >= 0
    free64 = o.run()[0] if cfg == 1 else None
    rows = []
    for fmt in fmts:
        views, labels, _ = PT.gpu_inputs(lf, fmt)
        ctx = lfd.Context(0)
        ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
        planes, lab, costs = ctx.plane_sweep(want_labels=True, want_costs=True)
        ctx.synchronize()
        labg = lab.cpu().numpy()[items]
        c = costs.cpu().numpy().astype(np.float64)[items][present]
        rel = np.abs(c - sw["cost"][present]) / np.maximum(np.abs(sw["cost"][present]), 1e-12)
        inside = PT.within(c, sw["cost_lo"][present], sw["cost_hi"][present])
        state = planes.cpu().numpy()
        out, _, _ = ctx.iterate(1, planes)
        ctx.synchronize()
        out = out.cpu().numpy()
        res = o.iterate(1, state.astype(np.float64), items=items)
        same = PT.same_plane(out[items], res["planes"][items])
        dep = np.abs(out[items, 0] - res["planes"][items, 0]) <= 5e-3 * np.maximum(res["planes"][items, 0], 1e-9)
        row = dict(fmt=fmt, sweep_label_identical=float(np.mean(labg[present] == sw["label"][present])),
                   cost_rel_err_median=float(np.median(rel)), cost_in_interval=float(inside.mean()),
                   iter1_identical=float(same.mean()), iter1_depth_0p5pct=float(dep.mean()))
        if free64 is not None:
            pf, _ = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
            ctx.synchronize()
            pf = pf.cpu().numpy()
            m = free64[:, 0] > 0
            row["free_flip_rate"] = float(1.0 - PT.same_plane(pf[m], free64[m]).mean())
            row["free_depth_0p5pct"] = float(np.mean(np.abs(pf[m, 0] - free64[m, 0]) <= 5e-3 * free64[m, 0]))
        rows.append(row)
        ctx.close()
    print(f"\nconfig {cfg} ({lf.name}), {n_items} sampled superpixels, oracle on the FP64 rendering:")
    for r in rows:
        print("  " + "  ".join(f"{k}={v:.4g}" if isinstance(v, float) else f"{k}={v}" for k, v in r.items()))
    for r in rows:
        assert r["sweep_label_identical"] >= LABEL_FLOOR
        assert r["iter1_depth_0p5pct"] >= DEPTH_FLOOR
        assert r["cost_rel_err_median"] <= COST_MEDIAN_MAX[r["fmt"]]
        if r["fmt"] in COST_INSIDE_MIN:
            assert r["cost_in_interval"] >= COST_INSIDE_MIN[r["fmt"]]
        if "free_depth_0p5pct" in r:
            assert r["free_depth_0p5pct"] >= FREE_DEPTH_FLOOR
