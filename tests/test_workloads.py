"""The synthetic workloads are what the documentation states: sizes, source counts,
source-pixel counts (the benchmark's denominator), patch rules, neighbour counts, and
the same draws for the same seed."""
import numpy as np
import pytest

from paper_1801_10277_gb300 import synth


def _patch_rule(prob):
    """Every patch lies inside its image; a patch away from the image edges is an odd
    square with a side in [15, 101] (the clamp of the generator's envelope rule)."""
    for n, x0, y0, w, h in prob.patches:
        H, W = prob.images[n].pixels.shape
        assert 0 <= x0 and 0 <= y0 and x0 + w <= W and y0 + h <= H and w >= 1 and h >= 1
        if 0 < x0 and 0 < y0 and x0 + w < W and y0 + h < H:
            assert w == h and w % 2 == 1 and 15 <= w <= 101, (n, x0, y0, w, h)


@pytest.mark.parametrize("cfg,name,n_src,n_img,shape,sp", [
    (0, "tiny_2src_5x48x48", 2, 5, (48, 48), 5930),
    (1, "field_500src_5x2048x1489", 500, 5, (1489, 2048), 1001730),
    (2, "crowded_64src_5x256x256", 64, 5, (256, 256), 109200),
    (4, "sweep_field_3125src_bright0.1", 3125, 5, (1489, 2048), 8629155),
])
def test_workload_sizes(cfg, name, n_src, n_img, shape, sp):
    p = synth.config(cfg)
    assert p.name == name and p.n_src == n_src and len(p.images) == n_img
    assert all(im.pixels.shape == shape for im in p.images)
    assert sorted(im.band for im in p.images) == [0, 1, 2, 3, 4]
    assert p.source_pixels() == sp
    _patch_rule(p)


def test_one_field_recipe():
    p = synth.config(1)
    gal = p.truth[:, synth.I_A + 1] > 0.5
    assert 0.5 < gal.mean() < 0.7                       # 60 % galaxies
    assert np.all(p.truth[:, 0] >= 0) and np.all(p.truth[:, 0] <= 2048)
    assert np.all(p.truth[:, 1] >= 0) and np.all(p.truth[:, 1] <= 1489)
    assert all(im.sky == 150.0 and im.calib == 0.005 for im in p.images)
    assert all(im.psf.shape == (3, 6) for im in p.images)   # 3 PSF components per band


def test_crowded_region_neighbour_counts():
    p = synth.config(2)
    deg = np.diff(p.nbr_offsets)
    assert deg.min() >= 2 and deg.max() <= 12


def test_same_seed_same_draws():
    a, b = synth.config(1), synth.config(1)
    np.testing.assert_array_equal(a.theta, b.theta)
    np.testing.assert_array_equal(a.patches, b.patches)
    for ia, ib in zip(a.images, b.images):
        np.testing.assert_array_equal(ia.pixels, ib.pixels)
    c = synth.config(1, seed=2028)
    assert not np.array_equal(a.theta, c.theta)
