"""Dense depth output (step a5): the depth maps of lfd_rasterize and
lfd_estimate against the oracle's rasteriser, pixel by pixel.

Section III-A asks for one depth map per view; every pixel takes the depth of
its superpixel's plane along the pixel ray (the D(p) of Eq. 10), camera z,
and 0 where the plane is missing or lies behind the camera there.

Tolerance, from the FP32 evaluation on the GPU: the inverse depth of pixel p
is g_r + g_0 dx + g_1 dy (dx, dy its offset from the superpixel's rounded
centroid, the three coefficients rounded once from FP64), two FMAs, then an
IEEE reciprocal.  With u = 2^-24 and cond = (|g_r| + |g_0 dx| + |g_1 dy|) /
|inverse depth| the relative error is at most u (3 cond + 2); the test allows
1.5 times that, which is below 1e-6 for every pixel with cond <= 3 (every
pixel of a fronto-parallel plane has cond = 1).  Validity (depth > 0) must
match wherever the oracle's inverse depth is further from 0 than that error.
"""
import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth
import parity as PT

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


def _error_bound(o, K, planes, V, H, W):
    """Per pixel (relative error bound, absolute inverse-depth error bound,
    inverse depth) of the GPU's FP32 evaluation.  The plane's inverse-depth
    vector g = K^-T n / (n . d K^-1 (c,1)) is formed here only to bound the
    rounding; the expected depths are the oracle's."""
    rel, absb, invs = [], [], []
    for v in range(V):
        Ki = np.linalg.inv(K[v])
        st = o.sp_stats(v)
        off, pix, cen = st["off"], st["pix"], st["cen"]
        rb = np.full(H * W, np.inf)
        ab = np.zeros(H * W)
        iv = np.zeros(H * W)
        for s in range(len(off) - 1):
            a, b = off[s], off[s + 1]
            pl = planes[o.sp_base[v] + s]
            if a == b or not pl[0] > 0:
                continue
            n = pl[1:4]
            rho = pl[0] * (n @ (Ki @ [cen[s, 0], cen[s, 1], 1.0]))
            if rho == 0:
                continue
            g = (Ki.T @ n) / rho
            rx, ry = np.rint(cen[s])
            p = pix[a:b]
            dx, dy = p % W - rx, p // W - ry
            gr = g[0] * rx + g[1] * ry + g[2]
            inv = gr + g[0] * dx + g[1] * dy
            mag = abs(gr) + np.abs(g[0] * dx) + np.abs(g[1] * dy)
            iv[p] = inv
            ab[p] = 3 * U * mag + U * np.abs(inv)
            with np.errstate(divide="ignore"):
                rb[p] = 1.5 * U * (3 * mag / np.abs(inv) + 2)
        rel.append(rb.reshape(H, W))
        absb.append(ab.reshape(H, W))
        invs.append(iv.reshape(H, W))
    return rel, absb, invs


def _compare_depth(o, K, planes, gpu_depth, report):
    V, H, W = gpu_depth.shape
    _, od = o.rasterize(planes.astype(np.float64))
    rel, absb, invs = _error_bound(o, K, planes.astype(np.float64), V, H, W)
    n_px = n_valid = n_checked = 0
    worst = 0.0
    for v in range(V):
        g = gpu_depth[v].astype(np.float64)
        ref = od[v]
        decided = np.abs(invs[v]) > 2 * absb[v]                   # validity not within the FP32 error
        vo, vg = ref > 0, g > 0
        assert np.array_equal(vo[decided], vg[decided]), f"view {v}: validity differs on decided pixels"
        assert np.all(g[~vg] == 0.0) and np.all(ref[~vo] == 0.0)   # invalid pixels are exactly 0
        both = vo & vg & np.isfinite(rel[v])
        err = np.abs(g[both] - ref[both]) / ref[both]
        assert np.all(err <= rel[v][both]), f"view {v}: max rel err {err.max():.3g}"
        well = both & (rel[v] <= 1.5 * U * 11)                     # cond <= 3
        assert np.all(np.abs(g[well] - ref[well]) <= 1e-6 * ref[well])
        n_px += g.size
        n_valid += int(vo.sum())
        n_checked += int(both.sum())
        worst = max(worst, float(err.max()) if err.size else 0.0)
    report.update(pixels=n_px, valid=n_valid, compared=n_checked, max_rel_err=worst)


def _slanted_state(o, rng, base):
    """Planes with random normals, about a third of them steep enough that
    part of the superpixel lies behind the camera, some missing."""
    st = base.copy()
    for gs in range(o.S_total):
        if st[gs, 0] <= 0:
            continue
        k = rng.integers(4)
        if k == 0:
            n = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), -1.0])     # steep: crosses the horizon
        elif k == 1:
            n = np.array([rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), -1.0])
        elif k == 2:
            st[gs] = 0.0                                                       # no plane
            continue
        else:
            continue
        st[gs, 1:] = n / np.linalg.norm(n)
    return st.astype(np.float32)


def test_rasterize_depth_matches_oracle_config1(lfd):
    lf = synth.make_config(1)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf)
    o = PT.make_oracle(lf, rgb, params)
    ctx = lfd.Context(0)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    sweep, _, _ = ctx.plane_sweep()
    ctx.synchronize()
    rng = np.random.default_rng(31)
    for name, st in (("sweep", sweep.cpu().numpy()), ("slanted", _slanted_state(o, rng, sweep.cpu().numpy()))):
        dep = ctx.rasterize(torch.from_numpy(st).cuda())
        ctx.synchronize()
        rep = {}
        _compare_depth(o, lf.rig.K, st, dep.cpu().numpy(), rep)
        print(f"depth parity config1 {name}:", rep)
        if name == "slanted":
            assert rep["valid"] < 0.8 * rep["pixels"]                  # missing planes and pixels behind the camera


def test_estimate_depth_out_matches_oracle_config2(lfd):
    """Full config-2 size through lfd_estimate (the call the bench times): the
    depth maps it writes equal the oracle's rasterisation of the planes it
    returns."""
    lf = synth.make_config(2, device="cuda")
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf)
    ctx = lfd.Context(0)
    planes, depth = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    ctx.synchronize()
    o = PT.make_oracle(lf, rgb, params)
    rep = {}
    _compare_depth(o, lf.rig.K, planes.cpu().numpy(), depth.cpu().numpy(), rep)
    print("depth parity config2 estimate:", rep)
    assert rep["valid"] > 0.9 * rep["pixels"]
