"""End to end on data drawn from the model itself: the expected image at a known truth
(celeste_render), Poisson counts around it, the Newton fit from the perturbed starts,
and the catalog scored against the truth.  The bright sources (r flux >= 10 nmgy,
signal-to-noise of tens or more) must come back close to the truth: positions within
0.1 px, r magnitudes and colours within 0.1 mag on average, no galaxy called a star."""
import copy

import numpy as np
import pytest

from paper_1801_10277_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def test_fit_recovers_truth_on_model_drawn_images(cel):
    prob = synth.config(1)
    truth = prob.truth.copy()
    star = truth[:, synth.I_A] >= 0.5
    truth[:, synth.I_A] = np.where(star, 0.995, 0.005)
    truth[:, synth.I_A + 1] = 1.0 - truth[:, synth.I_A]
    P = cel.Problem(prob)
    E, V = P.render(truth)
    assert all(np.all(e >= im.sky) for e, im in zip(E, prob.images))
    assert all(np.all(v >= 0) for v in V)
    P.close()
    rng = np.random.default_rng(17)
    pm = copy.copy(prob)
    pm.images = [copy.copy(im) for im in prob.images]
    for im, e in zip(pm.images, E):
        im.pixels = rng.poisson(e).astype(np.float32)
    Pm = cel.Problem(pm)
    th, it, st, el = Pm.fit(prob.theta, precision=cel.FP32, max_sweeps=3)
    assert el > Pm.elbo(prob.theta, precision=cel.FP64)[0]
    bright = np.exp(truth[:, synth.I_R1]) >= 10.0
    assert bright.sum() >= 100
    score = Pm.catalog_score(Pm.catalog(th)[bright], Pm.catalog(truth)[bright])
    assert score["position"] < 0.1, score
    assert score["brightness"] < 0.1, score
    for c in ("ug", "gr", "ri", "iz"):
        assert score[f"color_{c}"] < 0.1, score
    assert score["missed_gal"] == 0.0, score
    Pm.close()
