"""Synthetic accuracy and ablation suite (the analogues of the paper's
iteration-convergence and energy-term studies, Section IV): depth maps of the
rendered configurations against their ground truth, as bad-pixel rates
(relative inverse-depth error above 1 % and above 5 %), over the iteration
count, with each energy term switched off (term_mask: bit 0 smoothness
E_s of Eq. 5-7, bit 1 the consistency term E_c of Eq. 8 with its visibility and
occlusion parts, bit 2 the occlusion part O of Eq. 11 alone), and after depth
fusion (Section III-D).  Only flags of the C ABI are used."""
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


def _bad(depth, gt):
    """Shares of pixels with ground truth whose relative inverse-depth error exceeds 1 % / 5 %
    (a pixel without an estimate counts as bad)."""
    m = gt > 0
    est = depth[m]
    inv_err = np.where(est > 0, np.abs(1.0 / np.maximum(est, 1e-12) - 1.0 / gt[m]) * gt[m], np.inf)
    return float(np.mean(inv_err > 0.01)), float(np.mean(inv_err > 0.05))


@pytest.mark.parametrize("cfg", [1, 2])
def test_accuracy_over_iterations_terms_and_fusion(lfd, cfg):
    lf = synth.make_config(cfg, device="cuda")
    views, labels, _ = PT.gpu_inputs(lf, "rgba8")
    gt = lf.depth.cpu().numpy()
    base = synth.method_params(lf)
    ctx = lfd.Context(0)

    def run(**over):
        p = dict(base)
        p.update(over)
        _, depth = ctx.estimate(views, labels, lf.rig.K, lf.rig.R, lf.rig.t, lf.GW, lf.GH, p)
        ctx.synchronize()
        return depth

    rows = []
    n_it = base["iterations"]
    curve = []
    for it in range(0, n_it + 1):
        b1, b5 = _bad(run(iterations=it).cpu().numpy(), gt)
        curve.append((it, b1, b5))
    # term_mask bit 1 switches E_c (V and O together, Eq. 8); bit 2 only O inside it
    for name, mask in (("all terms", 7), ("no occlusion O", 3), ("no E_c (smoothness only)", 5),
                       ("no smoothness E_s", 6)):
        b1, b5 = _bad(run(term_mask=mask).cpu().numpy(), gt)
        rows.append((name, b1, b5))
    # flagged variant, not in the paper: random plane samples in the refinement step
    b1, b5 = _bad(run(perturb_samples=16, perturb_scale=0.05).cpu().numpy(), gt)
    rows.append(("+ 16 perturbation samples", b1, b5))
    depth = run()
    fused = ctx.fuse(depth)
    ctx.synchronize()
    rows.append(("all terms + fusion", *_bad(fused.cpu().numpy(), gt)))
    print(f"\nconfig {cfg} ({lf.name}): bad pixels (relative inverse-depth error > 1 % / > 5 %)")
    for it, b1, b5 in curve:
        print(f"  iterations {it}: {100 * b1:6.2f} % / {100 * b5:6.2f} %")
    for name, b1, b5 in rows:
        print(f"  {name:26s} {100 * b1:6.2f} % / {100 * b5:6.2f} %")
    # the refinement improves on the sweep, and the full energy is not worse than smoothness alone
    assert curve[-1][2] < curve[0][2]
    assert rows[0][2] <= rows[2][2] + 0.02
