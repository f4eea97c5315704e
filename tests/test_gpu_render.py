"""The model's expected image and variance (celeste_render) against the oracle's E and
Var maps (every pixel of every image, sky included), FP64: relative 1e-12."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def _check(cel, prob):
    _, _, oe, ov = Oracle(prob).elbo(prob.theta, maps=True)
    P = cel.Problem(prob)
    E, V = P.render(prob.theta)
    e = np.concatenate([x.ravel() for x in E])
    v = np.concatenate([x.ravel() for x in V])
    np.testing.assert_allclose(e, oe, rtol=1e-12)
    np.testing.assert_allclose(v, ov, rtol=1e-11, atol=1e-12 * np.abs(ov).max())
    # a render leaves the problem usable and its evaluations unchanged
    tot, _ = P.elbo(prob.theta, precision=cel.FP64)
    assert tot == pytest.approx(Oracle(prob).elbo(prob.theta)[0], rel=1e-10)
    P.close()


@pytest.mark.parametrize("cfg", [0, 2])
def test_render_matches_oracle(cel, cfg):
    _check(cel, synth.config(cfg))


def test_render_edge_cases(cel):
    """Clipped patches, a one-pixel patch, a source with no patch, a sky map, a rotated
    WCS."""
    th = np.stack([H.star_theta(1.0, 2.0), H.star_theta(20.0, 21.0, a_star=0.3),
                   H.star_theta(10.0, 10.0), H.star_theta(30.0, 5.0)])
    th[1, synth.I_AXIS] = 0.35
    patches = (np.array([0, 3, 8, 9, 9], np.int32),
               np.array([(0, 0, 0, 9, 11), (1, 0, 0, 17, 5), (4, 0, 0, 3, 1),
                         (0, 10, 12, 23, 20), (1, 10, 12, 22, 19), (2, 5, 5, 27, 27),
                         (3, 12, 14, 20, 18), (4, 13, 13, 19, 19),
                         (2, 10, 10, 1, 1)], np.int32))
    prob = H.problem(th, H=33, W=35, patches=patches, wcs=[0.98, -0.05, 0.05, 0.98, 0.7, -0.4])
    prob.images[2].sky_map = np.random.default_rng(3).uniform(120, 180, (33, 35)).astype(np.float32)
    _check(cel, prob)


def test_render_one_field_full_size(cel):
    _check(cel, synth.config(1))
