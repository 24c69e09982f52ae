"""The flagged perturbation variant of the refinement step (random planes
around the propagated plane, not in the paper) on the GPU against the
oracle, state-injected: every superpixel whose oracle choice is decided
(separated from the other candidates by more than the tolerance) gets the
same plane; the others get an admissible one."""
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


def _propagated(o, lfd, state, gs, m, it):
    """(depth at the own centroid, normal) after propagation choice m of superpixel gs."""
    v = int(np.searchsorted(o.sp_base, gs, side="right") - 1)
    s = gs - int(o.sp_base[v])
    if m == 0:
        return float(state[gs, 0]), state[gs, 1:].astype(np.float64)
    GW = o.GW[v]
    size, steps = o.kernel_params(v)
    off = lfd.kernel_offsets(size, steps, it)[m]
    j = int(o.sp_base[v]) + (s // GW + int(off[1])) * GW + (s % GW + int(off[0]))
    st = o.sp_stats(v)
    cj, cs = st["cen"][j - int(o.sp_base[v])], st["cen"][s]
    d = o.plane_depth(v, state[j].astype(np.float64), cj, cs[0], cs[1])
    return d, state[j, 1:].astype(np.float64)


@pytest.mark.parametrize("K,scale", [(8, 0.05), (24, 0.2)])
def test_perturbation_samples_match_oracle(lfd, K, scale):
    lf = synth.make_config(1)
    views, labels, rgb = PT.gpu_inputs(lf, "rgba8")
    params = synth.method_params(lf, perturb_samples=K, perturb_scale=scale)
    o = PT.make_oracle(lf, rgb, params)
    ctx = lfd.Context(0)
    ctx.set_input(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, params)
    planes, _, _ = ctx.plane_sweep()
    state = planes.cpu().numpy()
    for it in (1, 2, 3):
        st_t = torch.tensor(state, dtype=torch.float32, device="cuda")
        out, choice, _ = ctx.iterate(it, st_t, want_choice=True)
        ctx.synchronize()
        out, choice = out.cpu().numpy(), choice.cpu().numpy()
        res = o.iterate(it, state.astype(np.float64), cand_cap=1024)
        same = PT.same_plane(out, res["planes"])
        decided = np.zeros(o.S_total, bool)
        adm = same.copy()
        won = 0
        for gs in range(o.S_total):
            m_o, t_o = int(res["choice"][gs, 0]), int(res["choice"][gs, 1])
            won += t_o >= 8
            if m_o < 0:
                decided[gs] = True
                continue
            cand = res["cand"][gs]
            dec = PT.separated_best(cand[:, 0].copy(), cand[:, 1], cand[:, 2], m_o)
            if dec:
                ref = res["ref"][gs]
                E = np.concatenate([[cand[m_o, 0]], ref[:, 0]])
                lo = np.concatenate([[cand[m_o, 1]], ref[:, 1]])
                hi = np.concatenate([[cand[m_o, 2]], ref[:, 2]])
                dec = PT.separated_best(E.copy(), lo, hi, t_o + 1)
            decided[gs] = dec
            if not same[gs]:
                m_g, t_g = int(choice[gs, 0]), int(choice[gs, 1])
                ok = np.isfinite(cand[m_g, 1]) and PT.admissible(cand[m_g, 2], cand[np.isfinite(cand[:, 0]), 1])
                if ok and t_g >= 0:
                    d, n = _propagated(o, lfd, state, gs, m_g, it)
                    ref = o.refine_candidates(state.astype(np.float64), gs, d, n, it)
                    lo_all = np.concatenate([[cand[m_g, 1]], ref[np.isfinite(ref[:, 1]), 1]])
                    ok = np.isfinite(ref[t_g, 2]) and PT.admissible(ref[t_g, 2], lo_all)
                adm[gs] = ok
        print(f"\nK={K} scale={scale} iteration {it}: identical {same.mean():.4f}, decided {decided.mean():.4f}, "
              f"identical when decided {same[decided].mean():.4f}, admissible {adm.mean():.4f}, sample wins {won}")
        assert same[decided].all()
        assert adm.all()
        assert won > 0
        state = out
