"""Per-patch linearised world -> pixel maps on the GPU (celeste_problem_create_ex)
against the oracle: a crowded region with every patch's map perturbed (ELBO, locals,
gradients, Hessians, both precisions) and the deep stack at full size (480 images per
source, distorted maps linearised per source; sampled sources on their neighbour
closure).  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests.helpers import neighbour_closure
from tests.test_wcs_pins import _image_maps, _perturbed_maps

pytestmark = pytest.mark.gpu

TOL = {0: (1e-10, 1e-10, 1e-8, 1e-8), 1: (1e-5, 1e-5, 1e-4, 1e-4)}   # total, local, grad, hess


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_crowded_with_perturbed_patch_maps(cel):
    prob = synth.config(2)
    prob.patch_wcs = _perturbed_maps(prob, np.random.default_rng(6))
    orc = Oracle(prob)
    o_tot, o_loc = orc.elbo(prob.theta)
    which = np.arange(0, prob.n_src, 4).astype(np.int32)
    o_lh, o_gh, o_h = orc.derivs(prob.theta, which=which, hess=True)
    _, o_g, _ = orc.derivs(prob.theta)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        te, tl, tg, th = TOL[prec]
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        assert rel(tot, o_tot) <= te, (prec, tot, o_tot)
        assert np.max(np.abs(loc - o_loc) / np.abs(o_loc)) <= tl
        assert rel_l2(g, o_g) <= tg, (prec, rel_l2(g, o_g))
        _, _, h = P.hess(prob.theta, precision=prec)
        for k, s in enumerate(which):
            assert rel_l2(h[s], o_h[k]) <= th, (prec, s, rel_l2(h[s], o_h[k]))
    P.close()


def test_image_maps_per_patch_are_the_plain_problem(cel):
    prob = synth.config(2)
    P = cel.Problem(prob)
    ref = P.elbo_grad(prob.theta, precision=cel.FP64)
    P.close()
    prob.patch_wcs = _image_maps(prob)
    P = cel.Problem(prob)
    got = P.elbo_grad(prob.theta, precision=cel.FP64)
    P.close()
    assert got[0] == ref[0]
    np.testing.assert_array_equal(got[2], ref[2])


def test_singular_patch_map_rejected(cel):
    prob = synth.config(0)
    pw = _image_maps(prob)
    pw[3, 0:4] = [1.0, 2.0, 0.5, 1.0]
    prob.patch_wcs = pw
    with pytest.raises(cel.CelesteError) as e:
        cel.Problem(prob)
    assert e.value.status == cel.ERR_ARG


def test_deep_stack_full_size_sampled(cel):
    prob = synth.config(5)
    assert len(prob.images) == 480 and np.all(np.diff(prob.patch_offsets) == 480)
    sample = np.sort(np.random.default_rng(13).choice(prob.n_src, 6, replace=False))
    keep = neighbour_closure(prob, sample)
    sub = synth.subset(prob, keep)
    pos = np.searchsorted(keep, sample).astype(np.int32)
    o_l, o_g, _ = Oracle(sub).derivs(sub.theta, which=pos)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        _, tl, tg, _ = TOL[prec]
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        assert np.isfinite(tot)
        assert np.max(np.abs(loc[sample] - o_l) / np.abs(o_l)) <= tl, prec
        assert rel_l2(g[sample], o_g) <= tg, (prec, rel_l2(g[sample], o_g))
    P.close()
