"""Small problem builders shared by the tests (inputs only, no method arithmetic)."""
import math

import numpy as np

from paper_1801_10277_gb300 import synth


def psf_single(sigma=1.5, w=1.0, xi=(0.0, 0.0)):
    return np.array([[w, xi[0], xi[1], sigma ** 2, 0.0, sigma ** 2]])


def star_theta(x, y, flux=20.0, r2=1e-4, c2=1e-4, a_star=0.5):
    th = np.zeros(synth.NPARAM)
    th[0:2] = [x, y]
    th[synth.I_EDEV], th[synth.I_AXIS], th[synth.I_ANGLE], th[synth.I_SCALE] = 0.3, 0.6, 0.7, 2.0
    for i in range(2):
        th[synth.I_R1 + i] = math.log(flux)
        th[synth.I_R2 + i] = r2
        th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4] = [0.1, -0.2, 0.3, -0.1]
        th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4] = c2
        th[synth.I_K + 8 * i:synth.I_K + 8 * i + 8] = 1.0 / 8
    th[synth.I_A], th[synth.I_A + 1] = a_star, 1 - a_star
    return th


def problem(thetas, H=32, W=32, psfs=None, bands=(0, 1, 2, 3, 4), pixels=None, sky=150.0,
            calib=0.005, wcs=None, patches=None, seed=1, prior=None):
    """Images of H x W; each source's patch is the whole image unless given."""
    rng = np.random.default_rng(seed)
    thetas = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
    S = thetas.shape[0]
    images = []
    for n, b in enumerate(bands):
        psf = psfs[n] if psfs is not None else synth.draw_psf(rng)
        px = (pixels[n] if pixels is not None else
              rng.poisson(sky, size=(H, W)).astype(np.float32))
        images.append(synth.Image(band=b, pixels=np.asarray(px, np.float32), sky=sky,
                                  calib=calib,
                                  wcs=np.array([1, 0, 0, 1, 0, 0.0]) if wcs is None else np.asarray(wcs, float),
                                  psf=np.asarray(psf, float)))
    if patches is None:
        offs = [0]
        rows = []
        for s in range(S):
            for n in range(len(bands)):
                rows.append((n, 0, 0, W, H))
            offs.append(len(rows))
        po, pa = np.array(offs, np.int32), np.array(rows, np.int32)
    else:
        po, pa = patches
    no, nb = synth.make_neighbours(S, po, pa)
    exp_mix, dev_mix = synth.load_profiles()
    prior_star, prior_r, prior_c = synth.draw_priors(rng) if prior is None else prior
    return synth.Problem(images=images, exp_mix=exp_mix, dev_mix=dev_mix, prior_star=prior_star,
                         prior_r=prior_r, prior_c=prior_c, theta=thetas.copy(),
                         truth=thetas.copy(), patch_offsets=po, patches=pa, nbr_offsets=no,
                         nbrs=nb, name="test")


def neighbour_closure(prob, sample):
    """The sample and every neighbour of a sampled source (ascending ids): the
    sub-problem on which the sampled sources' local objectives are exact."""
    keep = set(int(s) for s in sample)
    for s in sample:
        keep.update(int(o) for o in prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]])
    return np.array(sorted(keep), np.int64)
