"""The allocation-free entry point (celeste_patch_elbo_grad_noalloc) gives the same
ELBO and gradient as the problem-based entry point (celeste_elbo_grad) for one
source confined to one patch.

This entry point exists for callers that cannot call cudaMalloc (their device memory
belongs to another allocator, or they must not allocate on the calling path); its
scratch is a fixed device array inside the library, shared by every call, so the test
also calls it twice in a row.  The file sorts last so a failure here comes after
every other test has run."""
import numpy as np
import pytest

from paper_1801_10277_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = {0: (1e-10, 1e-8), 1: (1e-5, 1e-4)}


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste as cel
    cel.load()
    th = H.star_theta(31.3, 26.8, a_star=0.35, r2=0.04, c2=0.02)
    th[synth.I_AXIS], th[synth.I_ANGLE], th[synth.I_SCALE] = 0.45, 0.9, 2.6
    x0, y0, w, h = 11, 7, 41, 37     # ragged: 41 x 37 = 1517 pixels, six 256-pixel items
    patches = (np.array([0, 1], np.int32), np.array([(0, x0, y0, w, h)], np.int32))
    prob = H.problem(th, H=60, W=70, bands=(3,), patches=patches,
                     wcs=[0.99, -0.04, 0.04, 0.99, 1.5, -2.0], seed=5)
    return torch, cel, prob, (x0, y0, w, h)


def test_noalloc_matches_problem_entry_point_on_two_calls():
    torch, cel, prob, (x0, y0, w, h) = _setup()
    P = cel.Problem(prob)
    im = prob.images[0]
    d_pix = torch.tensor(np.ascontiguousarray(im.pixels[y0:y0 + h, x0:x0 + w]), device="cuda")
    d_th = torch.tensor(prob.theta[0], dtype=torch.float64, device="cuda")
    for prec in (cel.FP64, cel.FP32):
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        te, tg = TOL[prec]
        results = []
        for _ in range(2):
            d_tot = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            d_loc = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            d_g = torch.full((44,), np.nan, dtype=torch.float64, device="cuda")
            cel.patch_elbo_grad_noalloc(im, prob.exp_mix, prob.dev_mix, prob.prior_star,
                                        prob.prior_r, prob.prior_c, (x0, y0, w, h), d_pix, d_th,
                                        d_tot, d_loc, d_g, precision=prec)
            torch.cuda.synchronize()
            results.append((d_tot.item(), d_loc.item(), d_g.cpu().numpy()))
        for t2, l2, g2 in results:
            assert abs(t2 - tot) <= te * abs(tot)
            assert abs(l2 - loc[0]) <= te * abs(loc[0])
            assert np.linalg.norm(g2 - g[0]) <= tg * np.linalg.norm(g[0])
    P.close()


def test_noalloc_rejects_patches_beyond_its_scratch():
    torch, cel, prob, _ = _setup()
    im = prob.images[0]
    d_pix = torch.zeros((10, 102), dtype=torch.float32, device="cuda")
    d_th = torch.tensor(prob.theta[0], dtype=torch.float64, device="cuda")
    d_g = torch.zeros(44, dtype=torch.float64, device="cuda")
    with pytest.raises(cel.CelesteError) as e:
        cel.patch_elbo_grad_noalloc(im, prob.exp_mix, prob.dev_mix, prob.prior_star,
                                    prob.prior_r, prob.prior_c, (0, 0, 102, 10), d_pix, d_th,
                                    None, None, d_g)
    assert e.value.status == cel.ERR_ARG
    assert "101" in str(e.value)


def _compare(torch, cel, prob, patch, sky=None):
    """Both precisions, the allocation-free call against celeste_elbo_grad on the same
    one-source problem; sky (a [H][W] float32 map of the whole image, or None) is passed
    to the allocation-free call as the patch's device sky map."""
    x0, y0, w, h = patch
    P = cel.Problem(prob)
    im = prob.images[0]
    d_pix = torch.tensor(np.ascontiguousarray(im.pixels[y0:y0 + h, x0:x0 + w]), device="cuda")
    d_sky = None if sky is None else torch.tensor(np.ascontiguousarray(sky[y0:y0 + h, x0:x0 + w]), device="cuda")
    d_th = torch.tensor(prob.theta[0], dtype=torch.float64, device="cuda")
    for prec in (cel.FP64, cel.FP32):
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        te, tg = TOL[prec]
        d_tot = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        d_loc = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        d_g = torch.full((44,), np.nan, dtype=torch.float64, device="cuda")
        cel.patch_elbo_grad_noalloc(im, prob.exp_mix, prob.dev_mix, prob.prior_star, prob.prior_r,
                                    prob.prior_c, patch, d_pix, d_th, d_tot, d_loc, d_g, d_sky_map=d_sky,
                                    precision=prec)
        torch.cuda.synchronize()
        assert abs(d_tot.item() - tot) <= te * abs(tot), (prec, d_tot.item(), tot)
        assert abs(d_loc.item() - loc[0]) <= te * abs(loc[0])
        assert np.linalg.norm(d_g.cpu().numpy() - g[0]) <= tg * np.linalg.norm(g[0])
    P.close()


def test_noalloc_with_a_device_sky_map():
    """A per-pixel sky (the image's sky map, indexed in the patch's frame)."""
    torch, cel, prob, patch = _setup()
    im = prob.images[0]
    yy, xx = np.mgrid[0:im.pixels.shape[0], 0:im.pixels.shape[1]]
    sky = (140.0 + 0.3 * xx + 0.2 * yy + 5.0 * np.sin(0.3 * xx) * np.cos(0.2 * yy)).astype(np.float32)
    im.sky_map = sky
    _compare(torch, cel, prob, patch, sky=sky)


def test_noalloc_at_its_largest_patch():
    """A 101 x 101 patch: every item and tile slot of the static scratch layout in use."""
    torch, cel, _, _ = _setup()
    th = H.star_theta(55.2, 49.7, a_star=0.4, r2=0.03, c2=0.02)
    th[synth.I_AXIS], th[synth.I_ANGLE], th[synth.I_SCALE] = 0.6, 1.3, 3.1
    patch = (3, 2, 101, 101)
    prob = H.problem(th, H=110, W=112, bands=(1,), patches=(np.array([0, 1], np.int32),
                                                           np.array([(0,) + patch], np.int32)),
                     wcs=[1.01, 0.03, -0.02, 0.98, -0.7, 1.2], seed=9)
    _compare(torch, cel, prob, patch)


def test_noalloc_rejects_a_bad_model():
    """The model is checked as by celeste_problem_create: a brightness-prior variance of
    zero and a zero colour-prior weight are CELESTE_ERR_ARG, not a NaN ELBO."""
    torch, cel, prob, (x0, y0, w, h) = _setup()
    im = prob.images[0]
    d_pix = torch.tensor(np.ascontiguousarray(im.pixels[y0:y0 + h, x0:x0 + w]), device="cuda")
    d_th = torch.tensor(prob.theta[0], dtype=torch.float64, device="cuda")
    d_g = torch.zeros(44, dtype=torch.float64, device="cuda")
    bad_r = np.array(prob.prior_r, dtype=np.float64, copy=True)
    bad_r.reshape(-1)[1] = 0.0
    bad_c = np.array(prob.prior_c, dtype=np.float64, copy=True)
    bad_c.reshape(2, -1, 21)[1, 3, 0] = 0.0
    for pr, pc in ((bad_r, prob.prior_c), (prob.prior_r, bad_c)):
        with pytest.raises(cel.CelesteError) as e:
            cel.patch_elbo_grad_noalloc(im, prob.exp_mix, prob.dev_mix, prob.prior_star, pr, pc,
                                        (x0, y0, w, h), d_pix, d_th, None, None, d_g)
        assert e.value.status == cel.ERR_ARG
