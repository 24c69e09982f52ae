"""Pins of the SLIC oracle (the segmentation step before the method, Section
III-A): CIELAB of reference colours, the grid as a fixed point on a uniform
image, and superpixels that do not cross a strong colour edge."""
import numpy as np

from oracle import oracle as orc
from paper_1812_06856_gb300 import synth


def test_cielab_of_reference_colours():
    assert np.allclose(orc.rgb_to_lab([1, 1, 1]), [100.0, 0.0, 0.0], atol=1e-4)   # matrix given to 7 digits
    assert np.allclose(orc.rgb_to_lab([0, 0, 0]), [0.0, 0.0, 0.0], atol=1e-9)
    # sRGB primaries in CIELAB (D65), published values
    assert np.allclose(orc.rgb_to_lab([1, 0, 0]), [53.2408, 80.0925, 67.2032], atol=5e-3)
    assert np.allclose(orc.rgb_to_lab([0, 1, 0]), [87.7347, -86.1827, 83.1793], atol=5e-3)
    assert np.allclose(orc.rgb_to_lab([0, 0, 1]), [32.2970, 79.1875, -107.8602], atol=5e-3)


def test_uniform_image_keeps_the_regular_grid():
    """No colour differences: every pixel takes the nearest cell centre, which
    is its own cell's when the cells are equal; the means are the centres."""
    W, H, GW, GH = 64, 48, 8, 6
    rgb = np.full((H, W, 3), 0.4)
    lab, c = orc.slic(rgb, GW, GH, m=10.0, iterations=5)
    ref, gw, gh = synth.grid_labels(W, H, 8.0, False)
    assert (gw, gh) == (GW, GH)
    assert np.array_equal(lab, ref)
    seeds = orc.slic_seeds(rgb, GW, GH)
    assert np.allclose(c, seeds)


def test_superpixels_follow_a_strong_colour_edge():
    W, H, GW, GH = 60, 40, 6, 4
    rgb = np.zeros((H, W, 3))
    rgb[:, :27] = [0.9, 0.1, 0.1]
    rgb[:, 27:] = [0.1, 0.2, 0.9]
    lab, c = orc.slic(rgb, GW, GH, m=5.0, iterations=10)
    for l in np.unique(lab):
        cols = np.nonzero((lab == l).any(axis=0))[0]
        assert cols.max() < 27 or cols.min() >= 27          # one side of the edge only
    grid, _, _ = synth.grid_labels(W, H, 10.0, False)
    assert not np.array_equal(lab, grid)                      # the edge moved the boundary cells


def _assign_pixel(centres_rel, m=8.0):
    """Assignment of pixel (2, 0) of a black 6x4 image in a 3x1 grid (cells 2
    px wide, 4 high; S = sqrt(6*4/3) = sqrt(8), (m/S)^2 = 8 for m = 8), the
    pixel inside cell 1 so that it compares all three centres.  centres_rel:
    per cell (dL, da, db, dx, dy) relative to the pixel's own Lab and xy."""
    rgb = np.zeros((4, 6, 3))
    lab0 = orc.rgb_to_lab([0.0, 0.0, 0.0])
    c = np.array([[*(lab0 + r[:3]), 2.0 + r[3], 0.0 + r[4]] for r in centres_rel])
    lab, fl = orc.slic_assign(rgb, 3, 1, c, m)
    return int(lab[0, 2]), int(fl[0, 2])


def test_slic_distance_hand_computed_three_centres():
    """D^2 = |dLab|^2 + (m/S)^2 |dxy|^2 by hand, on three centres:
      cell 0: dLab = (0, 3, 4), dxy = 0          -> 25
      cell 1: dLab = 0,         dxy = (2, 0)     -> 8 * 4 = 32
      cell 2: dLab = (4, 0, 0), dxy = (0.5, 0.5) -> 16 + 8 * 0.5 = 20
    so cell 2 wins, well apart from 25.  Each plausible slip picks another
    cell: m/S instead of (m/S)^2 (cell 1: 11.3), a dropped a/b term (cell 0:
    0), a dropped spatial term (cell 1: 0)."""
    lab, fl = _assign_pixel([(0, 3, 4, 0, 0), (0, 0, 0, 2, 0), (4, 0, 0, 0.5, 0.5)])
    assert (lab, fl) == (2, 0)


def test_slic_distance_hand_computed_exact_tie():
    """Cell 2 moved to dxy = (0.75, 0.75): 16 + 8 * 1.125 = 25, an exact tie
    with cell 0 (flagged; either cell may win).  A dropped L term (9) or S
    taken as the cell width (2: 16 + 16 * 1.125 = 34) breaks the tie."""
    lab, fl = _assign_pixel([(0, 3, 4, 0, 0), (0, 0, 0, 2, 0), (4, 0, 0, 0.75, 0.75)])
    assert fl == 1 and lab in (0, 2)
    # away from the tie the flag clears: cell 2 at 16 + 8 * 0.5 = 20
    lab, fl = _assign_pixel([(0, 3, 4, 0, 0), (0, 0, 0, 2, 0), (4, 0, 0, 0.5, 0.5)])
    assert fl == 0
