"""GPU catalog rows and the Table II error summary through the C ABI against the
oracle's plain FP64 definitions (oracle/catalog.py): FP64 throughout, so values agree
to a few ulps (relative 1e-13, absolute 1e-12 for values near zero), the type decision
exactly, and the error summary (different summation order) to 1e-12."""
import numpy as np
import pytest

from oracle import catalog as OC
from paper_1801_10277_gb300 import synth
from tests.test_catalog_pins import random_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def _close(a, b):
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-12)
    col = OC.FIELDS.index("is_star")
    np.testing.assert_array_equal(a[:, col], b[:, col])


@pytest.mark.parametrize("cfg", [0, 2, 1])
def test_catalog_matches_oracle(cel, cfg):
    prob = synth.config(cfg)
    P = cel.Problem(prob)
    for th in (prob.theta, prob.truth):
        _close(P.catalog(th), OC.catalog(th))
    P.close()


def test_catalog_random_and_edge_parameters(cel):
    """Random parameters over wide ranges, a_star exactly 1/2, angles far outside
    [0, pi), tiny and large variances, and a ragged last CTA (70 sources)."""
    prob = synth.config(2)
    rng = np.random.default_rng(8)
    th = np.stack([random_theta(rng) for _ in range(prob.n_src)])
    th[0, synth.I_A:synth.I_A + 2] = [0.5, 0.5]
    th[1, synth.I_ANGLE] = -1e3
    th[2, synth.I_ANGLE] = 0.0
    th[3, synth.I_R2:synth.I_R2 + 2] = [1e-12, 5.0]
    P = cel.Problem(prob)
    _close(P.catalog(th), OC.catalog(th))
    P.close()


def test_catalog_multi_epoch_full_size(cel):
    prob = synth.config(3)   # 20,000 sources
    P = cel.Problem(prob)
    _close(P.catalog(prob.theta), OC.catalog(prob.theta))
    P.close()


def test_catalog_device_bit_identical_and_errors(cel):
    import torch
    prob = synth.config(2)
    P = cel.Problem(prob)
    host = P.catalog(prob.theta)
    d_th = torch.tensor(prob.theta, dtype=torch.float64, device="cuda")
    d_cat = torch.zeros(prob.n_src, cel.CAT_NFIELD, dtype=torch.float64, device="cuda")
    P.catalog_device(d_th, d_cat)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    np.testing.assert_array_equal(d_cat.cpu().numpy(), host)
    bad = prob.theta.copy()
    bad[5, synth.I_R2] = 0.0
    with pytest.raises(cel.CelesteError) as e:
        P.catalog(bad)
    assert e.value.status == cel.ERR_ARG
    P.catalog_device(torch.tensor(bad, dtype=torch.float64, device="cuda"), d_cat)
    assert P.device_status() == cel.ERR_ARG
    P.catalog_device(d_th, d_cat)   # a clean call clears it
    assert P.device_status() == 0
    P.close()


def _score_close(a, b):
    for k in OC.SCORE_FIELDS:
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-13), (k, a[k], b[k])


def test_score_matches_oracle(cel):
    """The start catalog of the one-field workload against its truth, a perturbed copy,
    and the empty catalog."""
    prob = synth.config(1)
    P = cel.Problem(prob)
    truth = OC.catalog(prob.truth)
    start = P.catalog(prob.theta)
    _score_close(P.catalog_score(start, truth), OC.score(start, truth))
    rng = np.random.default_rng(4)
    other = start + rng.normal(0, 0.1, start.shape)
    other[:, OC.FIELDS.index("is_star")] = rng.integers(0, 2, len(other))
    _score_close(P.catalog_score(other, truth), OC.score(other, truth))
    empty = np.zeros((0, cel.CAT_NFIELD))
    assert all(v == 0.0 for v in P.catalog_score(empty, empty).values())
    P.close()
