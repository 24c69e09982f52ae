"""The C-ABI library loads, exports every entry point include/lfdepth.h
declares, agrees with the Python binding's struct layouts, and its host logic
(neighbour views, propagation-kernel offsets) matches the oracle's independent
implementations bit for bit.  No CUDA computation is run here."""
import os
import re

import ctypes
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1812_06856_gb300 import build as lfd_build
from paper_1812_06856_gb300 import synth
import helpers as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lfdepth.h")


@pytest.fixture(scope="module")
def lfd():
    lfd_build.build()
    from paper_1812_06856_gb300 import lfd as mod
    mod.load()
    return mod


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(lfd_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for must in ("lfd_create", "lfd_destroy", "lfd_set_input", "lfd_plane_sweep", "lfd_rasterize", "lfd_iterate",
                 "lfd_estimate", "lfd_estimate_host", "lfd_score", "lfd_synchronize"):
        assert must in names


def test_library_exports_every_declared_symbol(lfd):
    lib = ctypes.CDLL(lfd.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_and_defaults(lfd):
    lib = lfd.load()
    assert lib.lfd_version() == 2
    p = lfd.params_struct({})
    assert (p.T, p.alpha, p.eta, p.kernel_step_sp, p.term_mask, p.jitter) == (0.04, 0.1, 0.5, 5.0, 7, 1)
    assert lib.lfd_status_string(6) == b"device-side input check failed"
    o = lfd.BatchOptions()
    lib.lfd_batch_options_default(ctypes.byref(o))
    assert (o.autotune, o.graph, o.sweep_threads, o.sweep_persistent, o.prop_blocks, o.prop_persistent,
            o.prop_batch, o.order_bands, o.prop_coop) == (0, 0, 256, 1, 8, 1, 32, 16, 0)


@pytest.mark.parametrize("case", [(10, 2, 1), (10, 2, 2), (10, 2, 3), (10, 2, 7), (4, 8, 1), (54, 11, 1),
                                  (54, 11, 2), (54, 11, 6), (0, 0, 1), (67, 13, 1), (67, 13, 8), (12, 40, 1),
                                  (1, 0, 1), (3, 1, 2)])
def test_kernel_offsets_match_oracle(lfd, case):
    assert np.array_equal(lfd.kernel_offsets(*case), orc.kernel_offsets(*case))


def test_kernel_offsets_exhaustive_small(lfd):
    for size in range(0, 30):
        for steps in range(0, 12):
            for it in range(1, 9):
                assert np.array_equal(lfd.kernel_offsets(size, steps, it), orc.kernel_offsets(size, steps, it))


def _rigs():
    yield synth.line_rig(3, 0.1, 300, 320, 240)
    yield synth.grid_rig(4, 4, 0.08, 900, 64, 48)
    yield synth.grid_rig(3, 5, 0.1, 900, 64, 48)
    yield synth.arc_rig(8, 30.0, 5.0, 960, 64, 48)
    rng = np.random.default_rng(1)
    V = 11
    K = np.stack([H.K_pinhole(100, 64, 48)] * V)
    R = np.stack([H.random_rotation(rng, 20) for _ in range(V)])
    C = rng.normal(size=(V, 3))
    t = np.stack([-R[v] @ C[v] for v in range(V)])
    yield synth.Rig(K, R, t, 64, 48)


@pytest.mark.parametrize("maxk", [0, 1, 4, 8])
def test_neighbor_views_match_oracle(lfd, maxk):
    for rig in _rigs():
        V = rig.V
        got = lfd.neighbor_views(rig.K, rig.R, rig.t, rig.W, rig.H, maxk)
        lab = np.zeros((rig.H, rig.W), np.int32)
        img = np.zeros((rig.H, rig.W, 3))
        o = orc.Oracle(rig.K, rig.R, rig.t, [img] * V, [lab] * V, 1, 1, H.params(max_neighbor_views=maxk), threads=1)
        for v in range(V):
            assert list(got[v]) == list(o.neighbor_views(v)), (V, v)


def test_host_entry_points_reject_bad_arguments(lfd):
    lib = lfd.load()
    cams = lfd.make_cameras(np.stack([np.eye(3)]), np.stack([np.eye(3)]), np.zeros((1, 3)), 8, 8)
    out = (ctypes.c_int32 * 8)()
    assert lib.lfd_neighbor_views(cams, 1, 0, out, None) == 1          # fewer than 2 views
    assert lib.lfd_kernel_offsets(10, 2, 1, None, 0) == 9 + 8 * 2       # size query


def test_workspace_required_counts_every_per_pixel_buffer(lfd):
    """The HBM figure the budget and the server's admission use: at least the
    per-pixel buffers (24-B RGBA8 sampling texture, 16-B rasterised map, 4-B
    superpixel pixel list) and exactly linear in the number of equal views."""
    lib = lfd.load()
    lf1 = synth.make_config(1, scale=0.25)
    def req(V):
        K, R, t = lf1.rig.K[:1].repeat(V, 0), lf1.rig.R[:1].repeat(V, 0), lf1.rig.t[:1].repeat(V, 0)
        cams = lfd.make_cameras(K, R, t, lf1.rig.W, lf1.rig.H)
        gw = (ctypes.c_int32 * V)(*([lf1.GW] * V))
        gh = (ctypes.c_int32 * V)(*([lf1.GH] * V))
        lf = lfd.LightFieldC(V, 0, cams, None, None, None, gw, gh)
        out = ctypes.c_uint64()
        assert lib.lfd_workspace_required(1, ctypes.byref(lf), ctypes.byref(out)) == 0
        return out.value
    px = lf1.rig.W * lf1.rig.H
    assert req(2) >= 2 * px * (24 + 16 + 4)
    a, b, c = req(2), req(4), req(8)
    assert (c - b) >= 2 * (b - a) - 4096 and (c - b) <= 2 * (b - a) + 4096
    out = ctypes.c_uint64()
    assert lib.lfd_workspace_required(0, None, ctypes.byref(out)) == 1


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the no-device path")
def test_server_create_fails_cleanly_without_a_device(lfd):
    lib = lfd.load()
    h = ctypes.c_void_p()
    assert lib.lfd_server_create(ctypes.byref(h), 0, 0, 2) != 0
    assert not h.value
