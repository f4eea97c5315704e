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
