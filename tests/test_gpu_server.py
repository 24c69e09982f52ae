"""Serving form: the frame server gives each rig exactly what the plain calls
give (cold frame = lfd_estimate; warm frame = lfd_estimate from the rig's
previous planes with the warm schedule), whatever other rigs share the GPU
and whichever batch a frame joins; a warm-started batch equals separate
calls; state moves between servers; budget and queue bounds are enforced."""
import pytest
import torch

from paper_1812_06856_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfd():
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def rigs():
    """Three small moving rigs (quarter/eighth resolution), two keyframes each."""
    out = []
    for name, scale in (("A", 0.25), ("B", 0.2), ("C", 0.125)):
        r = synth.make_serving_rig(name, "cuda", keyframes=2, scale=scale)
        r.params["num_labels"] = 64
        out.append(r)
    return out


def _frame(r, f):
    k = r.keyframe_of(f)
    g = r.rigs[k]
    return dict(views=r.views[k], labels=r.labels, K=g.K, R=g.R, t=g.t, GW=r.GW, GH=r.GH)


def _out(r):
    S = r.V * r.GW * r.GH
    g = r.rigs[0]
    return (torch.zeros((S, 4), dtype=torch.float32, device="cuda"),
            torch.zeros((r.V, g.H, g.W), dtype=torch.float32, device="cuda"))


def _reference(lfd, r, frames, warm_iters=3, warm_off=3):
    """The plain calls the server must reproduce."""
    ctx = lfd.Context(0)
    res, prev = [], None
    for f in range(frames):
        fr = _frame(r, f)
        p = dict(r.params)
        if prev is not None:
            p.update(iterations=warm_iters, warm_iter_offset=warm_off)
        planes, depth = ctx.estimate(fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], p,
                                     warm=prev)
        ctx.synchronize()
        prev = planes.clone()
        res.append((planes.clone(), depth.clone()))
    return res


def _server(lfd, slots):
    srv = lfd.Server(0, 0, slots)
    srv.configure(3, 3, 8)
    return srv


def _serve(lfd, srv, schedule, rigs):
    """Submit (rig index, frame) pairs in order, each polled before the rig's next."""
    outs = {}
    for ri, f in schedule:
        r = rigs[ri]
        pl, dp = _out(r)
        fr = _frame(r, f)
        rid = srv.submit(ri, fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], r.params,
                         planes_out=pl, depth_out=dp)
        assert rid is not None
        outs[(ri, f)] = (rid, pl, dp)
    results = {}
    for key, (rid, pl, dp) in outs.items():
        res = srv.poll(rid, -1)
        assert res["status"] == 0 and res["done_ns"] >= res["submit_ns"]
        results[key] = (res, pl, dp)
    return results


def test_cold_then_warm_frames_match_plain_calls(lfd, rigs):
    r = rigs[0]
    ref = _reference(lfd, r, 3)
    srv = _server(lfd, 1)
    got = _serve(lfd, srv, [(0, 0), (0, 1), (0, 2)], rigs)
    for f in range(3):
        res, pl, dp = got[(0, f)]
        assert res["warm"] == (f > 0) and res["frame"] == f
        assert torch.equal(pl, ref[f][0]) and torch.equal(dp, ref[f][1])
    srv.close()


def test_rig_alone_equals_rig_in_a_mix(lfd, rigs):
    alone = _server(lfd, 1)
    a = _serve(lfd, alone, [(0, f) for f in range(3)], rigs)
    alone.close()
    for slots in (1, 2):
        mix = _server(lfd, slots)
        sched = []
        for f in range(3):
            for ri in (2, 0, 1):
                sched.append((ri, f))
        m = _serve(lfd, mix, sched, rigs)
        # frames queued while others ran were merged into batches of several rigs
        assert max(m[k][0]["batch"] for k in m) >= 2
        assert all(m[k][0]["start_ns"] >= m[k][0]["submit_ns"] for k in m)
        st = mix.stats()
        assert st["frames"] == len(sched) and st["batches"] < len(sched)
        for f in range(3):
            assert torch.equal(a[(0, f)][1], m[(0, f)][1])
            assert torch.equal(a[(0, f)][2], m[(0, f)][2])
        mix.close()


def test_max_batch_one_runs_frames_alone(lfd, rigs):
    srv = _server(lfd, 1)
    srv.set_max_batch(1)
    m = _serve(lfd, srv, [(ri, 0) for ri in range(3)] + [(ri, 1) for ri in range(3)], rigs)
    assert all(v[0]["batch"] == 1 for v in m.values())
    srv.close()


def test_warm_batch_equals_separate_calls(lfd, rigs):
    """lfd_estimate_batch_warm with a cold light field between two warm ones
    (the sweep leaves the warm views out) gives the separate calls' bits."""
    prev = []
    for r in rigs:
        ref = _reference(lfd, r, 1)
        prev.append(ref[0][0])
    ctx = lfd.Context(0)
    items, warm, expect = [], [], []
    for ri, r in enumerate(rigs):
        fr = _frame(r, 1)
        p = dict(r.params)
        w = None
        if ri != 1:
            p.update(iterations=3, warm_iter_offset=3)
            w = prev[ri]
        items.append(dict(views=fr["views"], labels=fr["labels"], K=fr["K"], R=fr["R"], t=fr["t"], GW=fr["GW"],
                          GH=fr["GH"], params=p))
        warm.append(w)
        c1 = lfd.Context(0)
        pl, dp = c1.estimate(fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], p, warm=w)
        c1.synchronize()
        expect.append((pl.clone(), dp.clone()))
        c1.close()
    planes, depths = ctx.estimate_batch(items, warm=warm)
    ctx.synchronize()
    base = 0
    for ri, r in enumerate(rigs):
        S = r.V * r.GW * r.GH
        assert torch.equal(planes[base:base + S], expect[ri][0])
        assert torch.equal(depths[ri], expect[ri][1])
        base += S
    ctx.close()


def test_state_export_import_continues_the_stream(lfd, rigs):
    s1 = _server(lfd, 1)
    r1 = _serve(lfd, s1, [(1, 0), (1, 1)], rigs)
    state = s1.export_state(1)
    r1b = _serve(lfd, s1, [(1, 2)], rigs)
    s1.close()
    s2 = _server(lfd, 2)
    _serve(lfd, s2, [(1, 5)], rigs)                  # any frame: makes the layout known
    s2.import_state(1, state)
    r2 = _serve(lfd, s2, [(1, 2)], rigs)
    assert torch.equal(r1b[(1, 2)][1], r2[(1, 2)][1])
    assert torch.equal(r1b[(1, 2)][2], r2[(1, 2)][2])
    s2.close()


def test_budget_and_queue_bounds(lfd, rigs):
    r = rigs[0]
    fr = _frame(r, 0)
    small = lfd.Server(0, 1 << 20, 1)
    with pytest.raises(lfd.LfdError) as e:
        small.submit(0, fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], r.params)
    assert e.value.status == lfd.LFD_ERR_BUDGET
    small.close()
    srv = lfd.Server(0, 0, 1)
    srv.configure(3, 3, 1)
    first = srv.submit(0, fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], r.params)
    assert first is not None
    assert srv.submit(0, fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], r.params) is None
    res = srv.poll(first, -1)
    assert res["frame"] == 0
    again = srv.submit(0, fr["views"], fr["labels"], fr["K"], fr["R"], fr["t"], fr["GW"], fr["GH"], r.params)
    assert again is not None and srv.poll(again, -1)["warm"] == 1
    with pytest.raises(lfd.LfdError):
        srv.poll(12345678, 0)
    srv.close()
