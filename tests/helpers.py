"""Small hand-built inputs for pin tests (cameras, images, label maps, states).

Input construction only: nothing here computes any part of the depth method.
"""
from __future__ import annotations

import math

import numpy as np

from paper_1812_06856_gb300 import synth


def K_pinhole(f, W, H):
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


def parallel_rig(xs, f, W, H, ys=None):
    """Parallel cameras (R = I) at centres (xs[k], ys[k], 0)."""
    V = len(xs)
    ys = ys if ys is not None else [0.0] * V
    K = np.stack([K_pinhole(f, W, H)] * V)
    R = np.stack([np.eye(3)] * V)
    t = np.stack([-np.array([xs[k], ys[k], 0.0]) for k in range(V)])
    return K, R, t


def grid_label_map(W, H, GW, GH):
    lab, gw, gh = synth.grid_labels(W, H, W / GW)
    assert (gw, gh) == (GW, GH)
    return lab


def params(**over):
    p = dict(d_min=1.0, d_max=5.0, num_labels=32, iterations=2,
             T=0.04, sigma=0.0, alpha=0.1, eta=0.5,
             kernel_size_init=0, kernel_step_sp=5.0, max_neighbor_views=8,
             depth_domain=0, jitter=1, term_mask=7, sweep_frame=0,
             seed=12345, lf_index=0, xy_eps=0.0, warm_iter_offset=0)
    p.update(over)
    return p


def fronto_state(S_total, d):
    st = np.zeros((S_total, 4))
    st[:, 0] = d
    st[:, 3] = -1.0
    return st


def colour_image_from_sp(lab, sp_colours):
    """RGB image where each pixel takes its superpixel's colour."""
    return np.asarray(sp_colours, dtype=np.float64)[lab]


def random_rotation(rng, max_deg):
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    a = math.radians(rng.uniform(-max_deg, max_deg))
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(a) * Kx + (1 - math.cos(a)) * Kx @ Kx
