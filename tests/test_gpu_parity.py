"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Section / equation numbers refer to the paper
(arXiv 1812.06856, Section III)."""
import numpy as np
import pytest
import torch

from paper_1812_06856_gb300 import synth
import parity as PT

pytestmark = pytest.mark.gpu

# a non-identical choice counts as the same plane up to a tie when the oracle
# admits it (its energy interval reaches the best one), its depth at the
# centroid is within 0.5 % and its normal within this angle of the oracle's
TIE_ANGLE_DEG = 2.0


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def cfg1():
    lf = synth.make_config(1)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf)
    o = PT.make_oracle(lf, rgb, params)
    return lf, views, labels, rgb, params, o


def bind(lfd, lf, views, labels, params):
    ctx = lfd.Context(0)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    return ctx


# ---------------------------------------------------------------------------
# step a1: superpixel lists and statistics (bit-exact lists)
# ---------------------------------------------------------------------------

def _check_superpixels(ctx, o, V):
    for v in range(V):
        g = ctx.get_superpixels(v)
        st = o.sp_stats(v)
        assert np.array_equal(g["off"], st["off"])
        assert np.array_equal(g["pix"], st["pix"])
        assert np.array_equal(g["stats"][:, 6].astype(np.int64), st["cnt"])
        ne = st["cnt"] > 0
        assert np.allclose(g["stats"][ne, 0:2], st["cen"][ne], rtol=2e-7, atol=1e-5)
        assert np.allclose(g["stats"][ne, 2:5], st["col"][ne], rtol=2e-7, atol=1e-7)
        assert np.allclose(g["stats"][:, 5], st["minw"], rtol=1e-5, atol=1e-6)
        assert list(g["neighbours"]) == list(o.neighbor_views(v))


def test_superpixels_grid_labels(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    ctx = bind(lfd, lf, views, labels, params)
    ctx.synchronize()
    _check_superpixels(ctx, o, lf.rig.V)


def test_superpixels_perturbed_and_scattered_labels(lfd):
    lf = synth.make_config(1, scale=0.5)
    rng = np.random.default_rng(5)
    lab0, GW, GH = synth.grid_labels(lf.rig.W, lf.rig.H, 9.0, perturb=True, seed=3)
    lab1 = rng.integers(0, GW * GH, size=lab0.shape).astype(np.int32)      # scattered (degenerate) superpixels
    lab2 = lab0.copy()
    lab2[lab2 == 5] = 6                                                   # an empty superpixel
    lf.labels = np.stack([lab0, lab1, lab2])
    lf.GW, lf.GH = GW, GH
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf)
    o = PT.make_oracle(lf, rgb, params)
    ctx = bind(lfd, lf, views, labels, params)
    ctx.synchronize()
    _check_superpixels(ctx, o, lf.rig.V)


# ---------------------------------------------------------------------------
# steps a2-a4: plane sweep (Eq. 1-2)
# ---------------------------------------------------------------------------

def _sweep_compare(lfd, lf, views, labels, params, o, report):
    ctx = bind(lfd, lf, views, labels, params)
    planes, lab, costs = ctx.plane_sweep(want_labels=True, want_costs=True)
    ctx.synchronize()
    planes, lab, costs = planes.cpu().numpy(), lab.cpu().numpy(), costs.cpu().numpy().astype(np.float64)
    sw = o.sweep(np.arange(o.S_total), want_costs=True)
    ne = sw["label"] >= 0
    floor = PT.tssd_abs_floor(o)[:, None] + PT.ABS
    ok = PT.within(costs[ne], sw["cost_lo"][ne], sw["cost_hi"][ne], absf=floor[ne])
    unfl = sw["cost_lo"][ne] == sw["cost_hi"][ne]
    err = PT.rel_err(costs[ne][unfl], sw["cost"][ne][unfl])
    same = lab == sw["label"]
    adm = np.array([same[i] or PT.admissible(sw["cost_lo"][i, lab[i]] * -1, -sw["cost_hi"][i]) for i in range(len(lab))])
    # decided: the oracle's arg-min is separated from every other label by more
    # than the tolerance; there the GPU must agree exactly
    decided = np.array([ne[i] and PT.separated_best(-sw["cost"][i], -sw["cost_hi"][i], -sw["cost_lo"][i], sw["label"][i])
                        for i in range(len(lab))])
    report.update(cost_ok=float(ok.mean()), cost_max_rel_err_unflagged=float(err.max()) if err.size else 0.0,
                  cost_flagged=float(1 - unfl.mean()), label_identical=float(same[ne].mean()),
                  label_admissible=float(adm[ne].mean()), decided=float(decided[ne].mean()),
                  identical_when_decided=float(same[decided].mean()) if decided.any() else 1.0)
    # the plane of the chosen label: depth 1/(1/d_max + (k+u) delta), normal (0,0,-1)
    for i in np.nonzero(same & ne)[0]:
        assert abs(planes[i, 0] - sw["planes"][i, 0]) <= 1e-6 * sw["planes"][i, 0]
    assert np.all(planes[~ne] == 0) and np.all(lab[~ne] == -1)
    return ok, same, adm, ne


def test_sweep_costs_and_labels_config1(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print("sweep parity config1:", rep)
    assert ok.all()
    # every label is the oracle's arg-min or a near-tie inside the oracle's bounds
    # (counted separately); where the oracle's choice is decided it is identical
    assert adm[ne].all()
    assert rep["identical_when_decided"] == 1.0


@pytest.mark.parametrize("fmt", ["rgba_f16", "rgba_bf16", "rgba_f32"])
def test_sweep_float_formats(lfd, fmt):
    lf = synth.make_config(1, scale=0.5)
    views, labels, rgb = PT.gpu_inputs(lf, fmt)
    params = synth.method_params(lf, num_labels=32)
    o = PT.make_oracle(lf, rgb, params)
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print(f"sweep parity {fmt}:", rep)
    assert ok.all() and adm[ne].all() and rep["identical_when_decided"] == 1.0


def test_sweep_world_frame_on_arc_rig(lfd):
    lf = synth.make_config(2, scale=0.25, views=3)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=48, sweep_frame=1)
    o = PT.make_oracle(lf, rgb, params)
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print("sweep parity world frame:", rep)
    assert ok.all() and adm[ne].all() and rep["identical_when_decided"] == 1.0


# ---------------------------------------------------------------------------
# per-hypothesis energy terms (Eq. 3-11)
# ---------------------------------------------------------------------------

def _queries(o, state, rng, n):
    qs = []
    items = rng.choice(o.S_total, size=n, replace=False)
    for gs in items:
        v = int(np.searchsorted(o.sp_base, gs, side="right") - 1)
        s = int(gs - o.sp_base[v])
        if state[gs, 0] <= 0:
            continue
        kind = rng.integers(3)
        if kind == 0:
            pl = state[gs]
        elif kind == 1:                      # a neighbour's plane re-expressed as (depth, normal)
            j = int(rng.integers(o.S_total))
            pl = state[j] if state[j, 0] > 0 else state[gs]
            pl = np.array([pl[0] * rng.uniform(0.97, 1.03), *pl[1:]])
        else:                                # random slanted plane
            n_ = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), -1.0])
            pl = np.array([state[gs, 0] * rng.uniform(0.9, 1.1), *(n_ / np.linalg.norm(n_))])
        qs.append((v, s, *np.asarray(pl, np.float32).astype(np.float64)))
    return qs


def _score_compare(lfd, ctx, o, state, qs, report, domain_note=""):
    from paper_1812_06856_gb300.lfd import terms_dict
    st_t = torch.tensor(state, dtype=torch.float32, device="cuda")
    g = ctx.score(st_t, qs)
    orr = o.score(state.astype(np.float32).astype(np.float64), qs)
    bad = []
    unfl_err = []
    nfl = 0
    for q, rec, r in zip(qs, g, orr):
        n = r["nviews"]
        t = terms_dict(rec, n)
        checks = [("E", t["E"], r["E_lo"], r["E_hi"]), ("Ec", t["Ec"], r["Ec_lo"], r["Ec_hi"]),
                  ("Es", t["Es"], r["Es"], r["Es"]), ("tssd", t["tssd"], r["tssd_lo"], r["tssd_hi"])]
        for k in range(n):
            checks += [("S", t["S"][k], r["S_lo"][k], r["S_hi"][k]), ("V", t["Vt"][k], r["V_lo"][k], r["V_hi"][k]),
                       ("O", t["O"][k], r["O_lo"][k], r["O_hi"][k])]
        for name, gv, lo, hi in checks:
            if not PT.within(gv, lo, hi):
                bad.append((q, name, gv, lo, hi))
        flagged = r["E_lo"] != r["E_hi"] or r["flag_tssd"]
        nfl += flagged
        if not flagged:
            unfl_err.append(max(PT.rel_err(t["E"], r["E"]), PT.rel_err(t["tssd"], r["tssd"]),
                                PT.rel_err(t["Es"], r["Es"])))
            if not np.array_equal(t["nvalid"], r["nvalid"]) or not np.array_equal(t["nx"], r["nx"]):
                bad.append((q, "counts", t["nvalid"], r["nvalid"], (t["nx"], r["nx"])))
    report.update(n=len(qs), flagged=nfl / max(len(qs), 1), max_rel_err_unflagged=float(max(unfl_err or [0])),
                  failures=len(bad))
    return bad


def test_score_terms_config1(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    ctx = bind(lfd, lf, views, labels, params)
    state = o.sweep()["planes"]
    rng = np.random.default_rng(7)
    qs = _queries(o, state, rng, 400)
    rep = {}
    bad = _score_compare(lfd, ctx, o, state, qs, rep)
    print("score parity config1:", rep, bad[:5])
    assert not bad


@pytest.mark.parametrize("over", [dict(depth_domain=1), dict(term_mask=3), dict(term_mask=5), dict(xy_eps=1e-3)])
def test_score_terms_variants(lfd, over):
    lf = synth.make_config(1, scale=0.5)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=32, **over)
    o = PT.make_oracle(lf, rgb, params)
    ctx = bind(lfd, lf, views, labels, params)
    state = o.sweep()["planes"]
    qs = _queries(o, state, np.random.default_rng(9), 150)
    rep = {}
    bad = _score_compare(lfd, ctx, o, state, qs, rep)
    print("score parity", over, rep, bad[:5])
    assert not bad


def test_score_terms_arc_rig(lfd):
    lf = synth.make_config(2, scale=0.3, views=4)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, num_labels=48)
    o = PT.make_oracle(lf, rgb, params)
    ctx = bind(lfd, lf, views, labels, params)
    state = o.sweep()["planes"]
    qs = _queries(o, state, np.random.default_rng(11), 300)
    rep = {}
    bad = _score_compare(lfd, ctx, o, state, qs, rep)
    print("score parity arc rig:", rep, bad[:5])
    assert not bad


# ---------------------------------------------------------------------------
# steps a5-a7: state-injected iterations (Section III-C, III-E)
# ---------------------------------------------------------------------------

def _iterate_compare(lfd, ctx, o, state_f32, it, items, report):
    st_t = torch.tensor(state_f32, dtype=torch.float32, device="cuda")
    out, choice, energy = ctx.iterate(it, st_t, want_choice=True)
    ctx.synchronize()
    out, choice, energy = out.cpu().numpy(), choice.cpu().numpy(), energy.cpu().numpy()
    state64 = state_f32.astype(np.float64)
    res = o.iterate(it, state64, items=items, cand_cap=1024)
    same = PT.same_plane(out[items], res["planes"][items])
    adm = same.copy()
    decided = np.zeros(len(items), bool)
    for k, gs in enumerate(items):
        cand = res["cand"][k]
        m_o, t_o = int(res["choice"][k, 0]), int(res["choice"][k, 1])
        if m_o < 0:
            decided[k] = True
            continue
        dec = PT.separated_best(cand[:, 0].copy(), cand[:, 1], cand[:, 2], m_o)
        if dec:
            ref = res["ref"][k]
            E = np.concatenate([[cand[m_o, 0]], ref[:, 0]])
            lo = np.concatenate([[cand[m_o, 1]], ref[:, 1]])
            hi = np.concatenate([[cand[m_o, 2]], ref[:, 2]])
            dec = PT.separated_best(E.copy(), lo, hi, t_o + 1)
        decided[k] = dec
    for k in np.nonzero(~same)[0]:
        gs = items[k]
        cand = res["cand"][k]
        valid = np.isfinite(cand[:, 0])
        m_g = int(choice[gs, 0])
        ok = m_g < cand.shape[0] and np.isfinite(cand[m_g, 1]) and PT.admissible(cand[m_g, 2], cand[valid, 1])
        t_g = int(choice[gs, 1])
        if ok and t_g >= 0:
            ref = o.refine_candidates(state64, gs, float(out[gs, 0]))
            base_lo = cand[m_g, 1]
            lo_all = np.concatenate([[base_lo], ref[np.isfinite(ref[:, 1]), 1]])
            ok = np.isfinite(ref[t_g, 2]) and PT.admissible(ref[t_g, 2], lo_all)
        adm[k] = ok
    dep_rel = np.abs(out[items, 0] - res["planes"][items, 0]) / np.maximum(res["planes"][items, 0], 1e-9)
    dep = dep_rel <= 5e-3
    cosang = np.clip(np.sum(out[items, 1:] * res["planes"][items, 1:], axis=1), -1.0, 1.0)
    ang = np.degrees(np.arccos(cosang))
    ang[res["planes"][items, 0] <= 0] = 0.0
    close = same | (adm & dep & (ang <= TIE_ANGLE_DEG))
    report.update(identical=float(same.mean()), admissible=float(adm.mean()), decided=float(decided.mean()),
                  identical_when_decided=float(same[decided].mean()) if decided.any() else 1.0,
                  depth_within_0p5pct=float(dep.mean()), same_or_close_tie=float(close.mean()),
                  nonidentical=int((~same).sum()),
                  nonidentical_max_depth_rel=float(dep_rel[~same].max()) if (~same).any() else 0.0,
                  nonidentical_max_angle_deg=float(ang[~same].max()) if (~same).any() else 0.0, n=len(items))
    return out, same, adm


def test_iterations_state_injected_config1(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    ctx = bind(lfd, lf, views, labels, params)
    planes, _, _ = ctx.plane_sweep()
    state = planes.cpu().numpy()
    items = np.arange(o.S_total, dtype=np.int32)
    for it in range(1, params["iterations"] + 1):
        rep = {}
        out, same, adm = _iterate_compare(lfd, ctx, o, state, it, items, rep)
        print(f"iteration {it} state-injected:", rep)
        assert adm.all()
        assert rep["identical_when_decided"] == 1.0
        assert rep["depth_within_0p5pct"] == 1.0
        state = out


def test_iterations_state_injected_with_split_tolerance(lfd):
    """With a relative tolerance on the X/Y split of Eq. 10/11 (xy_eps) consistent
    pixels no longer sit on the split; the same protocol holds."""
    lf = synth.make_config(1)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, xy_eps=1e-4)
    o = PT.make_oracle(lf, rgb, params)
    ctx = bind(lfd, lf, views, labels, params)
    planes, _, _ = ctx.plane_sweep()
    state = planes.cpu().numpy()
    items = np.arange(o.S_total, dtype=np.int32)
    for it in range(1, params["iterations"] + 1):
        rep = {}
        out, same, adm = _iterate_compare(lfd, ctx, o, state, it, items, rep)
        print(f"iteration {it} state-injected, xy_eps 1e-4:", rep)
        assert adm.all() and rep["identical_when_decided"] == 1.0 and rep["depth_within_0p5pct"] == 1.0
        state = out


def test_north_star_bar_pooled_over_state_injected_iterations(lfd):
    """The benchmark spec's bar, pooled over every state-injected iteration of
    config 1 (four iterations, 900 superpixels) and of its geometry cut into
    8-px and 5-px superpixels (two iterations each): the same chosen plane on
    at least 99.9 % of superpixel-iterations, and depth within 0.5 % on all
    the rest, each of which the oracle admits as a tie."""
    import dataclasses
    base = synth.make_config(1)
    cases = [(base, base.params["iterations"])]
    for pitch in (8.0, 5.0):
        labs = []
        for v in range(base.rig.V):
            lab, GW, GH = synth.grid_labels(base.rig.W, base.rig.H, pitch, True, seed=2000 + v)
            labs.append(lab)
        cases.append((dataclasses.replace(base, labels=np.stack(labs), GW=GW, GH=GH, pitch=pitch), 2))
    n = n_same = 0
    for lf, iters in cases:
        views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
        params = synth.method_params(lf, iterations=iters)
        o = PT.make_oracle(lf, rgb, params)
        ctx = bind(lfd, lf, views, labels, params)
        planes, _, _ = ctx.plane_sweep()
        state = planes.cpu().numpy()
        items = np.arange(o.S_total, dtype=np.int32)
        for it in range(1, iters + 1):
            rep = {}
            out, same, adm = _iterate_compare(lfd, ctx, o, state, it, items, rep)
            assert adm.all() and rep["depth_within_0p5pct"] == 1.0
            n += len(items)
            n_same += int(same.sum())
            state = out
        ctx.close()
    print(f"north_star bar pooled: {n_same} of {n} superpixel-iterations identical ({n_same / n:.5f})")
    assert n_same >= 0.999 * n


def test_estimate_equals_staged_and_is_deterministic(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    ctx = lfd.Context(0)
    p1, d1 = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    p2, d2 = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    ctx.synchronize()
    assert torch.equal(p1, p2) and torch.equal(d1, d2)
    # staged: sweep then iterations through the public per-step calls
    ctx2 = bind(lfd, lf, views, labels, params)
    pl, _, _ = ctx2.plane_sweep()
    for it in range(1, params["iterations"] + 1):
        pl, _, _ = ctx2.iterate(it, pl)
    dep = ctx2.rasterize(pl)
    ctx2.synchronize()
    assert torch.equal(pl, p1) and torch.equal(dep, d1)
    # host-memory entry point gives the same bits
    vh = views.cpu().pin_memory()
    lh = labels.cpu().pin_memory()
    ph = torch.zeros_like(p1, device="cpu").pin_memory()
    dh = torch.zeros_like(d1, device="cpu").pin_memory()
    ctx3 = lfd.Context(0)
    ctx3.estimate_host(vh, lh, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params, ph, dh)
    ctx3.synchronize()
    assert torch.equal(ph, p1.cpu()) and torch.equal(dh, d1.cpu())


def test_end_to_end_config1_free_running(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    ctx = lfd.Context(0)
    planes, depth = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    ctx.synchronize()
    g = planes.cpu().numpy()
    op, _ = o.run()
    same = PT.same_plane(g, op)
    close = np.abs(g[:, 0] - op[:, 0]) <= 5e-3 * np.maximum(op[:, 0], 1e-9)
    gt = synth.gt_planes(lf).reshape(-1, 4)
    m = gt[:, 0] > 0
    err_g = np.median(np.abs(1 / g[m, 0] - 1 / gt[m, 0]) * gt[m, 0])
    err_o = np.median(np.abs(1 / op[m, 0] - 1 / gt[m, 0]) * gt[m, 0])
    print(f"free-running config1: identical {same.mean():.4f} depth within 0.5% {close.mean():.4f} "
          f"median rel inverse-depth error gpu {err_g:.5f} oracle {err_o:.5f}")
    # free-running, FP32 near-ties that go the other way change later choices,
    # so planes drift apart in their last bits (identical 78 %); depths stay
    # within 0.5 % on 99.9 % (bound: 99.5 %) and the accuracy matches the
    # oracle's (0.472 % vs 0.467 %; bound: within 10 %)
    assert close.mean() >= 0.995
    assert abs(err_g - err_o) <= 0.1 * err_o


def test_config2_full_size_sampled_state_injected(lfd):
    """Full config-2 size (8 x 1024x768, 256 labels) in the launch configuration
    the bench times; the oracle scores a deterministic sample of superpixels."""
    lf = synth.make_config(2, device="cuda")
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf)
    ctx = bind(lfd, lf, views, labels, params)
    planes, lab, costs = ctx.plane_sweep(want_labels=True, want_costs=True)
    ctx.synchronize()
    o = PT.make_oracle(lf, rgb, params)
    rng = np.random.default_rng(2)
    items = np.sort(rng.choice(o.S_total, size=48, replace=False)).astype(np.int32)
    sw = o.sweep(items, want_costs=True)
    c = costs.cpu().numpy().astype(np.float64)[items]
    ok = PT.within(c, sw["cost_lo"], sw["cost_hi"], absf=PT.tssd_abs_floor(o, items)[:, None] + PT.ABS)
    labg = lab.cpu().numpy()[items]
    adm = [labg[i] == sw["label"][i] or PT.admissible(-sw["cost_lo"][i, labg[i]], -sw["cost_hi"][i])
           for i in range(len(items)) if sw["label"][i] >= 0]
    print(f"config2 sweep sample: costs ok {ok.mean():.5f} labels identical "
          f"{np.mean(labg == sw['label']):.4f} admissible {np.mean(adm):.4f}")
    assert ok.all() and all(adm)
    state = planes.cpu().numpy()
    rep = {}
    out, same, adm2 = _iterate_compare(lfd, ctx, o, state, 1, items[:24], rep)
    print("config2 iteration 1 sample:", rep)
    assert adm2.all() and rep["identical_when_decided"] == 1.0 and rep["depth_within_0p5pct"] == 1.0


def test_config3_full_size_sampled_state_injected(lfd):
    """The headline frame at full size (16 x 1920x1080 FP16, 256 labels; the
    translation-pair sweep of the 4 x 4 grid) in the launch configuration the
    bench times; the oracle scores a deterministic sample of superpixels on
    the same FP16 colours, the sweep and a state-injected iteration 1."""
    lf = synth.make_config(3, device="cuda")
    views, labels, rgb = PT.gpu_inputs(lf, "rgba_f16")
    params = synth.method_params(lf)
    ctx = bind(lfd, lf, views, labels, params)
    assert ctx.pair_form() == 2
    planes, lab, costs = ctx.plane_sweep(want_labels=True, want_costs=True)
    ctx.synchronize()
    o = PT.make_oracle(lf, rgb, params)
    rng = np.random.default_rng(3)
    items = np.sort(rng.choice(o.S_total, size=40, replace=False)).astype(np.int32)
    sw = o.sweep(items, want_costs=True)
    c = costs.cpu().numpy().astype(np.float64)[items]
    ok = PT.within(c, sw["cost_lo"], sw["cost_hi"], absf=PT.tssd_abs_floor(o, items)[:, None] + PT.ABS)
    labg = lab.cpu().numpy()[items]
    adm = [labg[i] == sw["label"][i] or PT.admissible(-sw["cost_lo"][i, labg[i]], -sw["cost_hi"][i])
           for i in range(len(items)) if sw["label"][i] >= 0]
    print(f"config3 sweep sample: costs ok {ok.mean():.5f} labels identical "
          f"{np.mean(labg == sw['label']):.4f} admissible {np.mean(adm):.4f}")
    assert ok.all() and all(adm)
    state = planes.cpu().numpy()
    rep = {}
    out, same, adm2 = _iterate_compare(lfd, ctx, o, state, 1, items[:20], rep)
    print("config3 iteration 1 sample:", rep)
    assert adm2.all() and rep["identical_when_decided"] == 1.0 and rep["depth_within_0p5pct"] == 1.0


# ---------------------------------------------------------------------------
# boundary behaviour
# ---------------------------------------------------------------------------

def test_invalid_inputs_are_reported(lfd, cfg1):
    lf, views, labels, rgb, params, o = cfg1
    ctx = lfd.Context(0)
    with pytest.raises(lfd.LfdError) as e:
        ctx.iterate(1, torch.zeros((10, 4), device="cuda"))
    assert e.value.status == 8                       # no light field bound
    bad = dict(params, d_min=5.0, d_max=1.0)
    with pytest.raises(lfd.LfdError) as e:
        ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, bad)
    assert e.value.status == 1
    small = lfd.Context(0, hbm_budget=1 << 20)
    with pytest.raises(lfd.LfdError) as e:
        small.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    assert e.value.status == 4                       # over the HBM budget
    lab_bad = labels.clone()
    lab_bad[1, 5, 7] = lf.GW * lf.GH + 3             # label outside the grid
    ctx.set_input(views, lab_bad, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    with pytest.raises(lfd.LfdError) as e:
        ctx.synchronize()
    assert e.value.status == 6 and "view 1" in str(e.value)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    ctx.synchronize()                                # status cleared, context usable


# ---------------------------------------------------------------------------
# superpixel sizes across the compiled slot classes: small (1-2 slots per lane),
# the largest staged class (10 slots) and superpixels beyond the staged 320
# pixels (streamed), on config 1's views with other grid pitches
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pitch", [5.0, 24.0, 40.0])
def test_sweep_and_iterations_across_superpixel_sizes(lfd, pitch):
    import dataclasses
    base = synth.make_config(1)
    W, H = base.rig.W, base.rig.H
    labs = []
    for v in range(base.rig.V):
        lab, GW, GH = synth.grid_labels(W, H, pitch, True, seed=1000 + v)
        labs.append(lab)
    lf = dataclasses.replace(base, labels=np.stack(labs), GW=GW, GH=GH, pitch=pitch)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, iterations=2)
    o = PT.make_oracle(lf, rgb, params)
    sizes = np.array([o.sp_stats(v)["cnt"] for v in range(lf.rig.V)]).ravel()
    rep = {}
    ok, same, adm, ne = _sweep_compare(lfd, lf, views, labels, params, o, rep)
    print(f"\npitch {pitch}: superpixel sizes {sizes.min()}..{sizes.max()}, sweep:", rep)
    assert ok.all() and adm[ne].all() and rep["identical_when_decided"] == 1.0
    ctx = bind(lfd, lf, views, labels, params)
    planes, _, _ = ctx.plane_sweep()
    state = planes.cpu().numpy()
    items = np.arange(o.S_total, dtype=np.int32)
    for it in (1, 2):
        rep = {}
        out, same, adm = _iterate_compare(lfd, ctx, o, state, it, items, rep)
        print(f"pitch {pitch} iteration {it} state-injected:", rep)
        assert adm.all() and rep["identical_when_decided"] == 1.0 and rep["depth_within_0p5pct"] == 1.0
        state = out
    if pitch >= 24.0:
        assert sizes.max() > 320          # the streamed path ran
    else:
        assert sizes.max() <= 64          # one- and two-slot classes
