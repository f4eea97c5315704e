"""Per-patch world -> pixel maps (multi-epoch images whose WCS is linearised at each
source, Section III's per-image metadata): the oracle pinned by exact invariances and
finite differences, and the input generator's linearisation by finite differences."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests import helpers as H


def _galaxy(x, y):
    th = H.star_theta(x, y, a_star=0.3)
    th[synth.I_AXIS], th[synth.I_ANGLE], th[synth.I_SCALE] = 0.45, 0.8, 2.5
    return th


def _one_source(wcs=(0.98, -0.05, 0.05, 0.98, 0.7, -0.4)):
    prob = H.problem(_galaxy(15.2, 14.7)[None], H=32, W=32, wcs=list(wcs))
    return prob


def _image_maps(prob):
    return np.stack([prob.images[int(p[0])].wcs for p in prob.patches]).astype(np.float64)


def test_image_maps_per_patch_change_nothing():
    prob = H.problem(np.stack([_galaxy(10.0, 11.0), _galaxy(16.0, 15.5)]), H=30, W=30)
    base = Oracle(prob)
    t0, l0 = base.elbo(prob.theta)
    f0, g0, h0 = base.derivs(prob.theta, hess=True)
    prob.patch_wcs = _image_maps(prob)
    o = Oracle(prob)
    t1, l1 = o.elbo(prob.theta)
    f1, g1, h1 = o.derivs(prob.theta, hess=True)
    assert t0 == t1
    np.testing.assert_array_equal(l0, l1)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(h0, h1)


def test_patch_translation_moves_the_source():
    """t_p = t + delta in every patch: A u + t + delta = A (u + A^-1 delta) + t."""
    prob = _one_source()
    delta = np.array([0.37, -0.61])
    pw = _image_maps(prob)
    pw[:, 4:6] += delta
    A = np.array(prob.images[0].wcs[:4]).reshape(2, 2)
    th = prob.theta.copy()
    th[0, 0:2] += np.linalg.solve(A, delta)
    t_ref, _ = Oracle(prob).elbo(th)
    prob.patch_wcs = pw
    t_pw, _ = Oracle(prob).elbo(prob.theta)
    assert t_pw == pytest.approx(t_ref, rel=1e-13)


def test_patch_rotation_rotates_position_and_shape():
    """A_p = A R(alpha): A R u + t places the source at R u, and A R W(phi) R^T A^T =
    A W(phi + alpha) A^T turns its ellipse by alpha."""
    prob = _one_source()
    alpha = 0.23
    R = np.array([[math.cos(alpha), -math.sin(alpha)], [math.sin(alpha), math.cos(alpha)]])
    A = np.array(prob.images[0].wcs[:4]).reshape(2, 2)
    pw = _image_maps(prob)
    AR = A @ R
    pw[:, 0:4] = AR.ravel()
    # keep the source inside the patch: place it where R u lands at the old position
    th = prob.theta.copy()
    th[0, 0:2] = np.linalg.solve(R, th[0, 0:2])
    ref = th.copy()
    ref[0, 0:2] = R @ th[0, 0:2]
    ref[0, synth.I_ANGLE] += alpha
    t_ref, _ = Oracle(prob).elbo(ref)
    prob.patch_wcs = pw
    t_pw, _ = Oracle(prob).elbo(th)
    assert t_pw == pytest.approx(t_ref, rel=1e-12)


def _perturbed_maps(prob, rng, a=0.02, t=0.3):
    pw = _image_maps(prob)
    pw[:, 0:4] += rng.normal(0, a, size=(pw.shape[0], 4))
    pw[:, 4:6] += rng.normal(0, t, size=(pw.shape[0], 2))
    return pw


def test_gradient_and_hessian_with_patch_maps_by_differences():
    prob = H.problem(np.stack([_galaxy(10.0, 11.0), _galaxy(16.0, 15.5)]), H=30, W=30)
    prob.patch_wcs = _perturbed_maps(prob, np.random.default_rng(4))
    o = Oracle(prob)
    f, g, h = o.derivs(prob.theta, hess=True)
    for s in range(2):
        for i in (0, 1, synth.I_AXIS, synth.I_ANGLE, synth.I_SCALE):
            step = 1e-5
            tp, tm = prob.theta.copy(), prob.theta.copy()
            tp[s, i] += step
            tm[s, i] -= step
            fd = (o.elbo(tp)[1][s] - o.elbo(tm)[1][s]) / (2 * step)
            assert fd == pytest.approx(g[s, i], rel=2e-6, abs=1e-6 * abs(f[s]) * 1e-3)
            gp, gm = o.derivs(tp)[1][s], o.derivs(tm)[1][s]
            np.testing.assert_allclose((gp - gm) / (2 * step), h[s, i], rtol=1e-4,
                                       atol=1e-6 * np.abs(h[s]).max())


def test_generator_linearisation_by_differences():
    prob_img = synth.Image(band=2, pixels=np.zeros((10, 10), np.float32), sky=100.0, calib=0.005,
                           wcs=np.array([0.99, -0.02, 0.03, 1.01, 5.0, -3.0]),
                           psf=np.array([[1.0, 0, 0, 1.5, 0, 1.5]]),
                           warp=(192.0, 192.0, 192.0, 0.4, -0.3, 0.25, 0.5))
    u0 = np.array([250.0, 80.0])
    w = synth.linearised_wcs(prob_img, u0)
    J = w[:4].reshape(2, 2)
    h = 1e-4
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        col = (synth.pixel_position_full(prob_img, u0 + e) - synth.pixel_position_full(prob_img, u0 - e)) / (2 * h)
        np.testing.assert_allclose(J[:, k], col, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(J @ u0 + w[4:6], synth.pixel_position_full(prob_img, u0), rtol=1e-14)
