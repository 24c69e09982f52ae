"""Shared helpers of the GPU parity tests: identical inputs for the CUDA path
and the oracle, and the comparison rules.

Comparison rules (tolerances of the per-hypothesis parity protocol):
  * integer / index work (superpixel lists, counts, labels of unambiguous
    arg-mins) is compared bit for bit;
  * a floating-point term passes when it lies inside the oracle's admissible
    interval [lo, hi] widened by REL * max(|lo|, |hi|) + ABS; the interval is a
    single value except where the oracle flagged a discrete decision (window
    edge, nearest-pixel rounding, X/Y split) within its margin;
  * a chosen plane passes when it is the oracle's plane, or when the oracle's
    interval of the GPU's choice reaches the best certain energy (a tie that
    FP32 may resolve either way).
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as orc
from paper_1812_06856_gb300 import synth

REL = 1e-4      # per-hypothesis relative tolerance of the path's floating-point terms
ABS = 1e-7      # absolute floor (terms near 0: V_i, O_i, a Gaussian far in its tail)
# Two candidates whose energies each carry an error up to REL can swap when
# their gap is below 2 REL; a GPU choice is an admissible tie when its upper
# bound reaches the best lower bound within that, plus 25 %.
TIE_REL = 2.5e-4
# Absolute floor of a truncated-SSD sum (Eq. 2), per pixel-view sample: the
# bilinear colour an FP32 implementation interpolates is within ~3 ulp of 1
# (1.8e-7 in [0,1] units) of the exact value, so an untruncated SSD, whose
# colour differences sum to at most sqrt(3 T) = 0.35, moves by at most
# 2 * 0.35 * 1.8e-7 = 1.3e-7.  A sum of costs that nearly match (a cost far
# below 1e-3 per sample) is bounded by this, not by REL.
TSSD_ABS_PER_SAMPLE = 1.3e-7


def tssd_abs_floor(o, items=None) -> np.ndarray:
    """Per superpixel (global index, or `items`): TSSD_ABS_PER_SAMPLE x its
    pixel-view samples (pixels x neighbour views)."""
    out = []
    for v in range(o.V):
        cnt = o.sp_stats(v)["cnt"].astype(np.float64)
        out.append(cnt * len(o.neighbor_views(v)) * TSSD_ABS_PER_SAMPLE)
    f = np.concatenate(out)
    return f if items is None else f[np.asarray(items)]


def gpu_inputs(lf: synth.LightField, fmt: str = "rgba8", device="cuda"):
    """(views tensor on device, labels tensor on device, float64 RGB the oracle sees)."""
    if fmt == "rgba8":
        q = synth.quantize_rgba8(lf.rgb)
        views = q.to(device)
        rgb = synth.rgba8_as_float(q)
    else:
        dt = {"rgba_f16": torch.float16, "rgba_bf16": torch.bfloat16, "rgba_f32": torch.float32}[fmt]
        views = synth.to_rgba_float(lf.rgb, dt).to(device)
        rgb = views[..., :3].to(torch.float64).cpu()
    labels = torch.from_numpy(np.ascontiguousarray(lf.labels)).to(device)
    return views, labels, rgb


def make_oracle(lf, rgb, params, threads=None):
    return orc.Oracle(*synth.oracle_inputs(lf, rgb), params, threads=threads)


def within(g, lo, hi, rel=REL, absf=ABS):
    g, lo, hi = np.asarray(g, float), np.asarray(lo, float), np.asarray(hi, float)
    lo2 = np.minimum(lo, hi)
    hi2 = np.maximum(lo, hi)
    tol = rel * np.maximum(np.abs(lo2), np.abs(hi2)) + absf
    return (g >= lo2 - tol) & (g <= hi2 + tol)


def rel_err(g, o, floor=1e-6):
    g, o = np.asarray(g, float), np.asarray(o, float)
    return np.abs(g - o) / np.maximum(np.abs(o), floor)


def same_plane(a, b, rel_d=2e-6, abs_n=2e-6):
    a, b = np.asarray(a, float), np.asarray(b, float)
    dd = np.abs(a[..., 0] - b[..., 0]) <= rel_d * np.maximum(np.abs(b[..., 0]), 1e-12)
    nn = np.all(np.abs(a[..., 1:] - b[..., 1:]) <= abs_n, axis=-1)
    return dd & nn


def separated_best(E, lo, hi, best):
    """The oracle's choice `best` is decided: its interval lies above every other
    valid candidate's interval by more than the tie tolerance.  E/lo/hi are
    arrays over candidates (-inf = not evaluated)."""
    valid = np.isfinite(E)
    valid[best] = False
    if not valid.any():
        return True
    top = np.max(hi[valid])
    return lo[best] > top + TIE_REL * abs(top) + ABS


def admissible(E_hi_choice, E_lo_all):
    """The choice's upper bound reaches the best lower bound (within TIE_REL)."""
    best_lo = np.max(E_lo_all)
    return E_hi_choice + TIE_REL * abs(best_lo) + ABS >= best_lo
