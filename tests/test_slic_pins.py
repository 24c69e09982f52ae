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
