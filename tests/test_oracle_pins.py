"""Pins of the CPU oracle to facts that do not come from the oracle itself:
closed forms, invariants, limits that reduce to library routines, quadrature of the
definitions, finite differences and brute-force enumeration.

Each test names the passage of the paper (Section III / IV-D, Table II notes) or the
reading it pins.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss
from scipy import stats
from scipy.special import gammaln

from oracle.oracle import Oracle, brightness, free_derivs, from_free, to_free, tr_solve
from paper_1801_10277_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def gh(n):
    """Probabilists' Gauss-Hermite nodes/weights normalised to N(0, 1)."""
    x, w = hermegauss(n)
    return x, w / w.sum()


# ----------------------------------------------------------------------------- data


def test_profile_mixtures_normalised_and_half_light():
    """Galaxy profile mixtures: unit flux, and half the flux inside r = 1 (the
    'scale' of Table II's notes is the effective, half-light radius)."""
    exp_mix, dev_mix = synth.load_profiles()
    for m in (exp_mix, dev_mix):
        w, nu = m[:, 0], m[:, 1]
        assert abs(w.sum() - 1.0) < 1e-12
        assert np.all(nu > 0)
        inside = np.sum(w * (1 - np.exp(-1.0 / (2 * nu))))
        assert abs(inside - 0.5) < 5e-3


# ----------------------------------------------------------------------------- profiles


def _grid(H, W):
    yy, xx = np.mgrid[0:H, 0:W]
    return xx.ravel().astype(float), yy.ravel().astype(float)


def test_star_profile_matches_library_normal():
    """Star: the PSF mixture centred at the source (Section III: F from the catalog
    and image metadata); compared with scipy's bivariate normal density."""
    psf = np.array([[0.6, 0.1, -0.05, 2.0, 0.3, 1.5], [0.4, -0.2, 0.1, 4.0, -0.5, 3.0]])
    th = H.star_theta(10.3, 12.7)
    p = H.problem(th, H=24, W=24, psfs=[psf] * 5)
    o = Oracle(p)
    x, y = _grid(24, 24)
    gs, _ = o.profiles(th, 0, x, y)
    ref = np.zeros_like(x)
    for a, xx, yy, sxx, sxy, syy in psf:
        ref += a * stats.multivariate_normal(mean=[10.3 + xx, 12.7 + yy],
                                             cov=[[sxx, sxy], [sxy, syy]]).pdf(np.c_[x, y])
    np.testing.assert_allclose(gs, ref, rtol=1e-12, atol=1e-300)


def _moments(g, x, y):
    m0 = g.sum()
    mx, my = (g * x).sum() / m0, (g * y).sum() / m0
    cxx = (g * (x - mx) ** 2).sum() / m0
    cxy = (g * (x - mx) * (y - my)).sum() / m0
    cyy = (g * (y - my) ** 2).sum() / m0
    return m0, mx, my, np.array([[cxx, cxy], [cxy, cyy]])


@pytest.mark.parametrize("rho,phi_deg,sigma", [(0.5, 30.0, 3.0), (0.3, 120.0, 4.0)])
def test_galaxy_profile_mass_mean_and_axes(rho, phi_deg, sigma):
    """Galaxy profile: unit mass; mean at the position plus the PSF offsets; second
    moments = PSF second moments + (mixture variance) x an ellipse whose major axis
    lies at the stated angle and whose axis ratio is e_axis (Table II notes)."""
    psf = np.array([[0.7, 0.2, -0.1, 1.2, 0.1, 1.0], [0.3, -0.1, 0.3, 2.5, 0.0, 2.0]])
    Hh = Ww = 160
    th = H.star_theta(80.2, 79.6)
    th[synth.I_AXIS], th[synth.I_ANGLE], th[synth.I_SCALE] = rho, math.radians(phi_deg), sigma
    th[synth.I_EDEV] = 0.0   # exponential: compact tails, moments converge on the grid
    p = H.problem(th, H=Hh, W=Ww, psfs=[psf] * 5)
    o = Oracle(p)
    x, y = _grid(Hh, Ww)
    _, gg = o.profiles(th, 0, x, y)
    m0, mx, my, C = _moments(gg, x, y)
    assert abs(m0 - 1) < 1e-6
    assert abs(mx - (80.2 + psf[:, 0] @ psf[:, 1])) < 1e-6
    assert abs(my - (79.6 + psf[:, 0] @ psf[:, 2])) < 1e-6
    # PSF mixture covariance (including the spread of the offsets)
    mxi = psf[:, 0] @ psf[:, 1:3]
    Cp = np.zeros((2, 2))
    for a, xx, yy, sxx, sxy, syy in psf:
        d = np.array([xx, yy]) - mxi
        Cp += a * (np.array([[sxx, sxy], [sxy, syy]]) + np.outer(d, d))
    exp_mix, _ = synth.load_profiles()
    nu_bar = exp_mix[:, 0] @ exp_mix[:, 1]
    G = (C - Cp) / nu_bar
    ev, evec = np.linalg.eigh(G)
    assert abs(math.sqrt(ev[1]) - sigma) < 1e-3 * sigma
    assert abs(math.sqrt(ev[0] / ev[1]) - rho) < 1e-3
    major = evec[:, 1]
    ang = math.degrees(math.atan2(major[1], major[0])) % 180.0
    assert abs(ang - phi_deg) < 0.05


def test_galaxy_half_light_radius():
    """Scale is the half-light radius: with a negligible PSF, half of the light of a
    circular galaxy falls within r = e_scale (Table II notes)."""
    psf = H.psf_single(0.05)
    Hh = Ww = 301
    for edev in (0.0, 1.0):
        th = H.star_theta(150.0, 150.0)
        th[synth.I_AXIS], th[synth.I_SCALE], th[synth.I_EDEV] = 1.0, 25.0, edev
        p = H.problem(th, H=Hh, W=Ww, psfs=[psf] * 5)
        o = Oracle(p)
        x, y = _grid(Hh, Ww)
        _, gg = o.profiles(th, 0, x, y)
        r = np.hypot(x - 150, y - 150)
        # flux inside radius 25 relative to the analytic total of 1
        frac = gg[r <= 25.0].sum()
        assert abs(frac - 0.5) < 0.02


def test_galaxy_star_limit_and_symmetries():
    """sigma -> 0 turns the galaxy profile into the star's; axis ratio 1 makes the
    angle irrelevant; angle and angle + pi are the same ellipse; e_dev mixes the two
    profiles linearly."""
    psf = np.array([[0.6, 0.1, -0.05, 2.0, 0.3, 1.5], [0.4, -0.2, 0.1, 4.0, -0.5, 3.0]])
    th = H.star_theta(12.0, 11.0)
    p = H.problem(th, H=24, W=24, psfs=[psf] * 5)
    o = Oracle(p)
    x, y = _grid(24, 24)
    t0 = th.copy()
    t0[synth.I_SCALE] = 1e-9
    gs, gg = o.profiles(t0, 0, x, y)
    np.testing.assert_allclose(gg, gs, rtol=1e-12, atol=1e-300)
    t1 = th.copy()
    t1[synth.I_AXIS] = 1.0
    t2 = t1.copy()
    t2[synth.I_ANGLE] += 1.234
    np.testing.assert_allclose(o.profiles(t1, 0, x, y)[1], o.profiles(t2, 0, x, y)[1], rtol=1e-12)
    t3 = th.copy()
    t3[synth.I_ANGLE] += math.pi
    np.testing.assert_allclose(o.profiles(th, 0, x, y)[1], o.profiles(t3, 0, x, y)[1], rtol=1e-11)
    ge = o.profiles(np.r_[th[:2], 0.0, th[3:]], 0, x, y)[1]
    gd = o.profiles(np.r_[th[:2], 1.0, th[3:]], 0, x, y)[1]
    e = 0.37
    gm = o.profiles(np.r_[th[:2], e, th[3:]], 0, x, y)[1]
    np.testing.assert_allclose(gm, (1 - e) * ge + e * gd, rtol=1e-12)


def test_wcs_maps_position_and_shape():
    """The affine WCS (image metadata Lambda_n, Section III) maps world position u to
    pixel A u + t, and the galaxy ellipse by A G A^T: a pure translation by t gives
    the same profile shifted; a 90-degree rotation turns angle phi into phi + 90."""
    psf = H.psf_single(1.2)
    th = H.star_theta(20.0, 18.0)
    th[synth.I_AXIS], th[synth.I_ANGLE], th[synth.I_SCALE] = 0.4, 0.3, 3.0
    x, y = _grid(40, 40)
    p = H.problem(th, H=40, W=40, psfs=[psf] * 5)
    base = Oracle(p).profiles(th, 0, x, y)[1]
    p2 = H.problem(th, H=40, W=40, psfs=[psf] * 5, wcs=[1, 0, 0, 1, 3.0, -2.0])
    th2 = th.copy()
    th2[0:2] = [17.0, 20.0]
    np.testing.assert_allclose(Oracle(p2).profiles(th2, 0, x, y)[1], base, rtol=1e-12)
    # rotation by 90 degrees about the origin, then shift back into the image
    p3 = H.problem(th, H=40, W=40, psfs=[psf] * 5, wcs=[0, -1, 1, 0, 38.0, 0.0])
    th3 = th.copy()
    th3[0:2] = [18.0, 18.0]    # -> pixel (38 - 18, 18) = (20, 18)
    th3[synth.I_ANGLE] = 0.3 - math.pi / 2
    np.testing.assert_allclose(Oracle(p3).profiles(th3, 0, x, y)[1], base, rtol=1e-10)


# ----------------------------------------------------------------------------- brightness


def _band_logs(logr, c):
    """log brightness of bands u g r i z from log r and the adjacent-band log ratios
    c_j = log(l_{j+1} / l_j) (Section III), walking outward from the r band."""
    lr = logr
    lg = lr - c[1]
    lu = lg - c[0]
    li = lr + c[2]
    lz = li + c[3]
    return [lu, lg, lr, li, lz]


def test_brightness_moments_by_quadrature():
    """E[l_b] and E[l_b^2] under q (log-normal r, independent Gaussian colours) by a
    5-D Gauss-Hermite product rule over (log r, c)."""
    rng = np.random.default_rng(0)
    x, w = gh(10)
    th = H.star_theta(0, 0)
    for i in range(2):
        th[synth.I_R1 + i] = rng.normal(1.0, 0.5)
        th[synth.I_R2 + i] = rng.uniform(0.01, 0.2)
        th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4] = rng.normal(0, 0.5, 4)
        th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4] = rng.uniform(0.01, 0.1, 4)
    for i in range(2):
        mu = np.r_[th[synth.I_R1 + i], th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4]]
        sd = np.sqrt(np.r_[th[synth.I_R2 + i], th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4]])
        Z = np.stack(np.meshgrid(*([x] * 5), indexing="ij"), -1).reshape(-1, 5)
        Wt = np.prod(np.stack(np.meshgrid(*([w] * 5), indexing="ij"), -1).reshape(-1, 5), 1)
        V = mu + sd * Z
        logs = _band_logs(V[:, 0], V[:, 1:].T)
        for b in range(5):
            El, El2 = brightness(th, b, i)
            l = np.exp(logs[b])
            assert abs(El - Wt @ l) < 1e-11 * El
            assert abs(El2 - Wt @ l ** 2) < 1e-10 * El2


# ----------------------------------------------------------------------------- KL


def _prior_identical(D=8, mean=(0.2, -0.1, 0.3, 0.0), var=(0.3, 0.2, 0.4, 0.25)):
    prior_c = np.zeros((2, D, 21))
    for i in range(2):
        for d in range(D):
            prior_c[i, d, 0] = 1.0 / D
            prior_c[i, d, 1:5] = mean
            prior_c[i, d, 5:] = np.diag(var).ravel()
    return prior_c


def test_kl_zero_at_prior():
    """KL(q || p) = 0 when q equals the prior (Eq. 1's entropy and prior terms cancel)."""
    prior_r = np.array([[1.1, 0.7], [0.4, 1.3]])
    prior_c = _prior_identical()
    th = H.star_theta(5, 5, a_star=0.4)
    for i in range(2):
        th[synth.I_R1 + i], th[synth.I_R2 + i] = prior_r[i]
        th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4] = prior_c[i, 0, 1:5]
        th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4] = np.diag(prior_c[i, 0, 5:].reshape(4, 4))
        th[synth.I_K + 8 * i:synth.I_K + 8 * i + 8] = prior_c[i, :, 0]
    p = H.problem(th, H=8, W=8, prior=(0.4, prior_r, prior_c))
    assert abs(Oracle(p).kl(th[None])[0]) < 1e-14


def test_kl_brute_force_enumeration():
    """KL of the joint q(a) q(r|a) q(k|a) q(c|a) against p(a) p(r|a) p(k) p(c|a,k),
    enumerated over a and k with exact Gauss-Hermite rules over log r and c (the
    log-densities are quadratic, so 3 nodes per dimension are exact), densities from
    scipy."""
    rng = np.random.default_rng(3)
    _, prior_r, prior_c = synth.draw_priors(rng)
    for i in range(2):
        for d in range(8):
            A = rng.normal(0, 0.3, (4, 4))
            prior_c[i, d, 5:] = (A @ A.T + 0.2 * np.eye(4)).ravel()
            prior_c[i, d, 0] = rng.uniform(0.5, 1.5)
        prior_c[i, :, 0] /= prior_c[i, :, 0].sum()
    th = H.star_theta(5, 5, a_star=0.35)
    for i in range(2):
        th[synth.I_R1 + i], th[synth.I_R2 + i] = rng.normal(1, 0.3), rng.uniform(0.1, 0.5)
        th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4] = rng.normal(0, 0.4, 4)
        th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4] = rng.uniform(0.05, 0.3, 4)
        k = rng.uniform(0.2, 1, 8)
        th[synth.I_K + 8 * i:synth.I_K + 8 * i + 8] = k / k.sum()
    p = H.problem(th, H=8, W=8, prior=(0.4, prior_r, prior_c))
    kl = Oracle(p).kl(th[None])[0]
    x, w = gh(3)
    Z = np.stack(np.meshgrid(*([x] * 4), indexing="ij"), -1).reshape(-1, 4)
    Wc = np.prod(np.stack(np.meshgrid(*([w] * 4), indexing="ij"), -1).reshape(-1, 4), 1)
    pa = [0.4, 0.6]
    tot = 0.0
    for i in range(2):
        a = th[synth.I_A + i]
        r1, r2 = th[synth.I_R1 + i], th[synth.I_R2 + i]
        lr = r1 + math.sqrt(r2) * x
        qr = stats.norm(r1, math.sqrt(r2)).logpdf(lr)
        pr = stats.norm(prior_r[i, 0], math.sqrt(prior_r[i, 1])).logpdf(lr)
        c1 = th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4]
        c2 = th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4]
        cs = c1 + np.sqrt(c2) * Z
        qc = stats.multivariate_normal(c1, np.diag(c2)).logpdf(cs)
        for d in range(8):
            kd = th[synth.I_K + 8 * i + d]
            pc = stats.multivariate_normal(prior_c[i, d, 1:5], prior_c[i, d, 5:].reshape(4, 4)).logpdf(cs)
            # E over r and c of log q - log p for the joint atom (a = i, k = d)
            e_r = w @ (qr - pr)
            e_c = Wc @ (qc - pc)
            tot += a * kd * (math.log(a / pa[i]) + e_r + math.log(kd / prior_c[i, d, 0]) + e_c)
    assert abs(kl - tot) < 1e-10 * max(1.0, abs(tot))


# ----------------------------------------------------------------------------- E, V, ll


def _single_source(th, Hh=15, Ww=15, psf=None, sky=150.0):
    psf = H.psf_single(1.4) if psf is None else psf
    return H.problem(th, H=Hh, W=Ww, psfs=[psf] * 5, sky=sky)


def test_expected_rate_and_variance_by_quadrature():
    """E[F] and Var[F] of a pixel (Section III: F is the sky plus the source's light)
    from the joint q(a) q(l | a) by Gauss-Hermite quadrature, given the profiles."""
    th = H.star_theta(7.2, 6.9, a_star=0.3, r2=0.15, c2=0.05)
    th[synth.I_R1:synth.I_R1 + 2] = [math.log(30.0), math.log(45.0)]
    p = _single_source(th)
    o = Oracle(p)
    _, _, E, V = o.elbo(th[None], maps=True)
    x, w = gh(10)
    Z = np.stack(np.meshgrid(*([x] * 5), indexing="ij"), -1).reshape(-1, 5)
    Wt = np.prod(np.stack(np.meshgrid(*([w] * 5), indexing="ij"), -1).reshape(-1, 5), 1)
    xx, yy = _grid(15, 15)
    iota = 1.0 / 0.005
    off = 0
    for n, im in enumerate(p.images):
        gs, gg = o.profiles(th, n, xx, yy)
        m1 = np.zeros_like(xx)
        m2 = np.zeros_like(xx)
        for i, g in enumerate((gs, gg)):
            a = th[synth.I_A + i]
            mu = np.r_[th[synth.I_R1 + i], th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4]]
            sd = np.sqrt(np.r_[th[synth.I_R2 + i], th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4]])
            Vv = mu + sd * Z
            l = np.exp(_band_logs(Vv[:, 0], Vv[:, 1:].T)[im.band])
            El, El2 = Wt @ l, Wt @ l ** 2
            m1 += a * iota * El * g
            m2 += a * iota ** 2 * El2 * g * g
        np.testing.assert_allclose(E[off:off + 225], 150.0 + m1, rtol=1e-12)
        np.testing.assert_allclose(V[off:off + 225], m2 - m1 ** 2, rtol=1e-9, atol=1e-9)
        off += 225


def test_delta_method_against_quadrature_of_elog():
    """The reading of E_q[log F]: log E - Var / (2 E^2), the second-order Taylor
    (delta-method) expansion of log F about E[F].  Against Gauss-Hermite quadrature
    of E_q[log F] on a single source of certain type: the remainder must be the next
    Taylor term mu3 / (3 E^3) up to the fourth-order term mu4 / (4 E^4), with the
    central moments mu_k of F also taken by quadrature; at zero variance both are
    log F exactly."""
    for r2 in (1e-10, 0.01, 0.05):
        th = H.star_theta(7.0, 7.0, a_star=0.5, r2=r2, c2=1e-12)
        th[synth.I_A], th[synth.I_A + 1] = 1 - 1e-13, 1e-13
        th[synth.I_R1:synth.I_R1 + 2] = math.log(200.0)
        p = _single_source(th)
        o = Oracle(p)
        _, _, E, V = o.elbo(th[None], maps=True)
        xx, yy = _grid(15, 15)
        gs, _ = o.profiles(th, 2, xx, yy)  # r band: brightness = r
        x, w = gh(80)
        iota = 200.0
        l = np.exp(th[synth.I_R1] + math.sqrt(r2) * x)
        F = 150.0 + iota * np.outer(gs, l)          # [pixels][nodes]
        Elog = np.log(F) @ w
        Eq = F @ w
        mu3 = ((F - Eq[:, None]) ** 3) @ w
        mu4 = ((F - Eq[:, None]) ** 4) @ w
        E2, V2 = E[2 * 225:3 * 225], V[2 * 225:3 * 225]
        approx = np.log(E2) - V2 / (2 * E2 ** 2)
        resid = Elog - approx
        assert np.all(np.abs(resid - mu3 / (3 * E2 ** 3)) <= mu4 / (2 * E2 ** 4) + 1e-13)
        if r2 < 1e-8:
            assert np.abs(resid).max() < 1e-12


def test_poisson_special_case():
    """With vanishing brightness variances and a certain type, the expected
    log-likelihood is the Poisson log-pmf (Section III: x ~ Poisson(F)) up to the
    log x! constant the ELBO drops."""
    th = H.star_theta(7.0, 7.0, a_star=1 - 1e-12, r2=1e-14, c2=1e-14)
    th[synth.I_A] = 1 - 1e-12
    th[synth.I_A + 1] = 1e-12
    p = _single_source(th)
    o = Oracle(p)
    tot, loc, E, V = o.elbo(th[None], maps=True)
    kl = o.kl(th[None])[0]
    x = np.concatenate([im.pixels.ravel() for im in p.images]).astype(float)
    ll = stats.poisson.logpmf(x, E) + gammaln(x + 1)
    assert abs((tot + kl) - ll.sum()) < 1e-9 * abs(ll.sum())


def test_total_flux_approaches_brightness():
    """Summed over a growing patch, E[F] - sky approaches iota * sum_i a_i E[l_i]
    (profiles carry unit mass)."""
    th = H.star_theta(40.0, 40.0, a_star=0.4, r2=0.05, c2=0.02)
    th[synth.I_SCALE] = 2.5
    th[synth.I_EDEV] = 0.0
    prev = None
    for side in (21, 41, 81):
        off = (81 - side) // 2
        patches = (np.array([0, 5], np.int32),
                   np.array([(n, off, off, side, side) for n in range(5)], np.int32))
        p = H.problem(th, H=81, W=81, psfs=[H.psf_single(1.3)] * 5, patches=patches)
        o = Oracle(p)
        _, _, E, _ = o.elbo(th[None], maps=True)
        flux = (E[:81 * 81] - 150.0).sum()
        El0, _ = brightness(th, 0, 0)
        El1, _ = brightness(th, 0, 1)
        target = 200.0 * (th[synth.I_A] * El0 + th[synth.I_A + 1] * El1)
        err = abs(flux - target) / target
        if prev is not None:
            assert err <= prev + 1e-15
        prev = err
    assert prev < 1e-6


def test_elbo_total_equals_sum_of_locals_when_disjoint():
    """Total ELBO over the union of patches = sum of local objectives when patches
    do not overlap (block coordinate ascent, Section IV-D)."""
    ths = np.stack([H.star_theta(6.0, 6.0), H.star_theta(25.0, 25.0)])
    patches = (np.array([0, 5, 10], np.int32),
               np.array([(n, 0, 0, 13, 13) for n in range(5)] +
                        [(n, 18, 18, 14, 14) for n in range(5)], np.int32))
    p = H.problem(ths, H=32, W=32, patches=patches)
    tot, loc = Oracle(p).elbo(ths)
    assert abs(tot - loc.sum()) < 1e-9 * abs(tot)


# ----------------------------------------------------------------------------- derivatives


def test_gradient_and_hessian_finite_differences(cfg0):
    """Central differences of the local ELBO (value code) against the jet gradient,
    and of the jet gradient against the jet Hessian, for all 44 parameters."""
    o = Oracle(cfg0)
    th = cfg0.theta.copy()
    _, g, h = o.derivs(th, hess=True)
    for s in range(cfg0.n_src):
        fd = np.zeros(44)
        fdh = np.zeros((44, 44))
        for j in range(44):
            e = 1e-6 * max(1.0, abs(th[s, j]))
            a, b = th.copy(), th.copy()
            a[s, j] += e
            b[s, j] -= e
            fd[j] = (o.elbo(a)[1][s] - o.elbo(b)[1][s]) / (2 * e)
            ga = o.derivs(a, which=[s])[1][0]
            gb = o.derivs(b, which=[s])[1][0]
            fdh[:, j] = (ga - gb) / (2 * e)
        assert np.linalg.norm(fd - g[s]) <= 1e-6 * np.linalg.norm(g[s])
        assert np.linalg.norm(fdh - h[s]) <= 1e-6 * np.linalg.norm(h[s])
        assert np.abs(h[s] - h[s].T).max() <= 1e-12 * np.abs(h[s]).max()


def test_round_galaxy_angle_gradient_zero():
    """Axis ratio 1: the ELBO cannot depend on the angle, so d/d angle = 0 and so is
    every second derivative through the angle except the mixed one with the axis
    ratio (the angle matters again as soon as the ratio leaves 1)."""
    th = H.star_theta(8.0, 8.0, a_star=0.3)
    th[synth.I_AXIS] = 1.0
    p = _single_source(th, 17, 17)
    _, g, h = Oracle(p).derivs(th[None], hess=True)
    assert abs(g[0, synth.I_ANGLE]) < 1e-9 * np.abs(g[0]).max()
    row = np.delete(h[0, synth.I_ANGLE], synth.I_AXIS)
    assert np.abs(row).max() < 1e-9 * np.abs(h[0]).max()


def test_unconstrained_map_round_trip_and_jacobian(cfg0):
    th = cfg0.theta[1]
    t = to_free(th)
    back, J = from_free(t, jac=True)
    np.testing.assert_allclose(back, th, rtol=1e-12, atol=1e-14)
    for a in range(41):
        e = 1e-6
        tp, tm = t.copy(), t.copy()
        tp[a] += e
        tm[a] -= e
        fd = (from_free(tp) - from_free(tm)) / (2 * e)
        np.testing.assert_allclose(J[:, a], fd, rtol=1e-6, atol=1e-9)
    # sum-to-one constraints hold in the image of the map
    assert abs(back[synth.I_A] + back[synth.I_A + 1] - 1) < 1e-15
    for i in range(2):
        assert abs(back[synth.I_K + 8 * i:synth.I_K + 8 * i + 8].sum() - 1) < 1e-14


def test_free_map_keeps_underflowing_weights_normal(cfg0):
    """A colour-component logit far below the others (its softmax weight underflows):
    the map keeps the weight at or above 1e-120, so the local objective's derivatives in
    the 44 parameters and in the 41 free coordinates stay finite, and the free gradient
    along that logit vanishes (d k / d t = k (1 - k) ~ 1e-120).  Away from underflow
    the weights are the softmax itself."""
    o = Oracle(cfg0)
    s = 1
    th = cfg0.theta.copy()
    t = to_free(th[s])
    ks = slice(synth.I_K, synth.I_K + 8)
    ex = np.exp(np.append(t[27:34], 0.0))
    np.testing.assert_allclose(from_free(t)[ks], ex / ex.sum(), rtol=1e-15, atol=0)
    t[27 + 3] = -800.0   # exp(-800) is 0 in FP64
    x = from_free(t)
    assert np.all(x[ks] >= 1e-120) and x[synth.I_K + 3] < 1.01e-120
    th[s] = x
    _, g, h = o.derivs(th, which=[s], hess=True)
    assert np.isfinite(g).all() and np.isfinite(h).all()
    gt, ht = free_derivs(t, g[0], h[0])
    assert np.isfinite(gt).all() and np.isfinite(ht).all()
    assert abs(gt[27 + 3]) < 1e-100 * np.abs(gt).max()


def test_free_derivatives_match_finite_differences(cfg0):
    """Gradient / Hessian in the 41 unconstrained coordinates (chain rule through the
    map) against central differences of ELBO_s(theta(t))."""
    o = Oracle(cfg0)
    s = 1
    th = cfg0.theta.copy()
    t = to_free(th[s])
    _, g, h = o.derivs(th, which=[s], hess=True)
    gt, ht = free_derivs(t, g[0], h[0])

    def f(tt):
        x = th.copy()
        x[s] = from_free(tt)
        return o.elbo(x)[1][s]

    def grad(tt):
        x = th.copy()
        x[s] = from_free(tt)
        _, gg, hh = o.derivs(x, which=[s], hess=True)
        return free_derivs(tt, gg[0], hh[0])[0]

    fd = np.zeros(41)
    fdh = np.zeros((41, 41))
    for a in range(41):
        e = 1e-6
        tp, tm = t.copy(), t.copy()
        tp[a] += e
        tm[a] -= e
        fd[a] = (f(tp) - f(tm)) / (2 * e)
        fdh[:, a] = (grad(tp) - grad(tm)) / (2 * e)
    assert np.linalg.norm(fd - gt) <= 1e-6 * np.linalg.norm(gt)
    assert np.linalg.norm(fdh - ht) <= 1e-5 * np.linalg.norm(ht)


# ----------------------------------------------------------------------------- trust region


def _kkt(c, B, delta, p):
    """Global optimality of the trust-region step (More & Sorensen): some lambda >= 0
    with (B + lambda I) p = -c, lambda (delta - |p|) = 0, B + lambda I PSD."""
    n = len(c)
    r = -c - B @ p
    pn = np.linalg.norm(p)
    lam = float(r @ p) / float(p @ p) if pn > 0 else 0.0
    assert pn <= delta * (1 + 1e-10)
    assert np.linalg.norm(r - lam * p) <= 1e-8 * (np.linalg.norm(c) + np.linalg.norm(B) * pn)
    assert lam >= -1e-10 * np.linalg.norm(B)
    if lam > 1e-10 * np.linalg.norm(B):
        assert abs(pn - delta) <= 1e-10 * delta
    assert np.linalg.eigvalsh(B + lam * np.eye(n)).min() >= -1e-9 * np.linalg.norm(B)


def test_trust_region_subproblem_cases():
    rng = np.random.default_rng(5)
    n = 41
    A = rng.normal(size=(n, n))
    Q, _ = np.linalg.qr(A)
    # interior: PD, large radius -> Newton step
    lam = rng.uniform(1, 10, n)
    B = Q @ np.diag(lam) @ Q.T
    c = rng.normal(size=n)
    p, pn = tr_solve(c, B, 1e6)
    np.testing.assert_allclose(p, -np.linalg.solve(B, c), rtol=1e-10, atol=1e-12)
    # boundary, PD
    p, pn = tr_solve(c, B, 0.05)
    _kkt(c, B, 0.05, p)
    # indefinite
    lam2 = lam.copy()
    lam2[:5] = -rng.uniform(1, 5, 5)
    B2 = Q @ np.diag(lam2) @ Q.T
    p, pn = tr_solve(c, B2, 0.7)
    _kkt(c, B2, 0.7, p)
    # hard case: c orthogonal to the lowest eigenvector
    i0 = int(np.argmin(lam2))
    c3 = c - (Q[:, i0] @ c) * Q[:, i0]
    p, pn = tr_solve(c3, B2, 5.0)
    _kkt(c3, B2, 5.0, p)


# ----------------------------------------------------------------------------- fit


def test_colouring_is_proper_and_greedy(cfg0):
    from paper_1801_10277_gb300.synth import crowded_region
    p = crowded_region()
    col, nc = Oracle(p).colouring()
    for s in range(p.n_src):
        nb = p.nbrs[p.nbr_offsets[s]:p.nbr_offsets[s + 1]]
        assert np.all(col[nb] != col[s])
        lower = set(col[nb[nb < s]].tolist())
        assert col[s] == min(set(range(nc + 1)) - lower)


def test_fit_recovers_truth_on_noiseless_image():
    """Trust-region Newton (Section IV-D) on an image equal to the model's expected
    counts at the truth, with nearly flat priors: converges in tens of iterations
    (Section IV-D) to the truth's position and flux."""
    truth = H.star_theta(12.3, 11.6, a_star=0.99, r2=1e-4, c2=1e-4)
    truth[synth.I_R1:synth.I_R1 + 2] = math.log(40.0)
    psf = np.array([[0.7, 0.0, 0.0, 1.8, 0.1, 1.6], [0.3, 0.1, -0.1, 4.5, 0.0, 4.0]])
    flat_r = np.array([[math.log(40.0), 1e6], [math.log(40.0), 1e6]])
    flat_c = _prior_identical(var=(1e6, 1e6, 1e6, 1e6))
    prior = (0.5, flat_r, flat_c)
    p0 = H.problem(truth, H=25, W=25, psfs=[psf] * 5, prior=prior)
    _, _, E, _ = Oracle(p0).elbo(truth[None], maps=True)
    pix = [E[n * 625:(n + 1) * 625].reshape(25, 25) for n in range(5)]
    p = H.problem(truth, H=25, W=25, psfs=[psf] * 5, prior=prior, pixels=pix)
    start = truth.copy()
    start[0:2] += [0.4, -0.35]
    start[synth.I_R1:synth.I_R1 + 2] += math.log(1.2)
    start[synth.I_R2:synth.I_R2 + 2] = 0.05
    o = Oracle(p)
    th, it, st, el, sw = o.fit(start[None], max_sweeps=1)
    assert st[0] == 0
    assert it[0] <= 50
    assert np.abs(th[0, 0:2] - truth[0:2]).max() < 1e-4
    # the identifiable brightness: expected r-band flux sum_i a_i E[l_i]; the ELBO's
    # optimum keeps a little variance and type entropy, so allow 1 %
    flux = sum(th[0, synth.I_A + i] * brightness(th[0], 2, i)[0] for i in range(2))
    assert abs(flux / 40.0 - 1) < 1e-2
    # stationarity in the free coordinates, relative to the objective's scale
    f, g, h = o.derivs(th, hess=True)
    gt, _ = free_derivs(to_free(th[0]), g[0], h[0])
    assert np.abs(gt).max() < 1e-7 * abs(f[0])


def test_oracle_matches_its_stored_values():
    """Regression guard: the oracle reproduces the values make_oracle_golden.py stored
    (to summation-order rounding), so a change of its arithmetic is deliberate."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_two_source_oracle.json")
    with open(path) as f:
        ref = json.load(f)
    prob = synth.config(0)
    orc = Oracle(prob)
    tot, loc = orc.elbo(prob.theta)
    _, g, _ = orc.derivs(prob.theta)
    assert abs(tot - ref["elbo_total"]) <= 1e-12 * abs(ref["elbo_total"])
    assert np.allclose(loc, ref["elbo_local"], rtol=1e-12, atol=0)
    assert np.allclose(g, ref["grad"], rtol=1e-10, atol=1e-10)


def test_brute_force_three_by_three_star():
    """A star on 3 x 3 images with every term written out by hand: the Gaussian PSF
    at integer pixel centres, band brightness moments from the colour definition
    (log l_{j+1} = log l_j + c_j, walked out from the r band), E[F] and Var[F] of
    Section III's rate, and the expected log-likelihood x (log E - Var / (2 E^2)) - E
    summed over the pixels; the oracle's total ELBO plus its KL must equal the sum."""
    sig, ux, uy = 0.9, 1.2, 0.9
    th = H.star_theta(ux, uy, flux=30.0, r2=0.05, c2=0.02, a_star=1 - 1e-13)
    th[synth.I_A], th[synth.I_A + 1] = 1 - 1e-13, 1e-13
    p = H.problem(th, H=3, W=3, psfs=[H.psf_single(sig)] * 5, sky=150.0)
    o = Oracle(p)
    tot, loc = o.elbo(th[None])
    kl = o.kl(th[None])[0]
    r1, r2 = th[synth.I_R1], th[synth.I_R2]
    c1 = th[synth.I_C1:synth.I_C1 + 4]
    c2 = th[synth.I_C2:synth.I_C2 + 4]
    # log-brightness mean and variance per band u g r i z, from r outwards
    mean = [0.0] * 5
    var = [0.0] * 5
    mean[2], var[2] = r1, r2
    for b in (1, 0):                      # l_b = l_{b+1} / exp(c_b)
        mean[b], var[b] = mean[b + 1] - c1[b], var[b + 1] + c2[b]
    for b in (3, 4):                      # l_b = l_{b-1} exp(c_{b-1})
        mean[b], var[b] = mean[b - 1] + c1[b - 1], var[b - 1] + c2[b - 1]
    iota = 1.0 / 0.005
    a = th[synth.I_A]
    want = 0.0
    for im in p.images:
        b = im.band
        El = math.exp(mean[b] + var[b] / 2)
        El2 = math.exp(2 * mean[b] + 2 * var[b])
        for row in range(3):
            for col in range(3):
                g = math.exp(-((col - ux) ** 2 + (row - uy) ** 2) / (2 * sig * sig)) / (2 * math.pi * sig * sig)
                E = 150.0 + a * iota * El * g
                V = a * iota * iota * El2 * g * g - (a * iota * El * g) ** 2
                x = float(im.pixels[row, col])
                want += x * (math.log(E) - V / (2 * E * E)) - E
    assert abs((tot + kl) - want) <= 1e-11 * abs(want)
    assert abs((loc[0] + kl) - want) <= 1e-11 * abs(want)


def test_flux_stationarity_condition_of_an_isolated_star():
    """With vanishing brightness variances and a certain type the ELBO is the Poisson
    log-likelihood sum x log F - F minus the KL, so its derivative in the log flux r1
    is sum (x / F - 1) iota E[l] g minus the KL's, and the KL's is
    a_star (r1 - prior mean) / prior variance (Gaussian KL in the mean): the oracle's
    gradient entry against that closed form at two fluxes."""
    sig, ux, uy = 1.1, 6.3, 5.8
    for flux in (25.0, 60.0):
        th = H.star_theta(ux, uy, flux=flux, r2=1e-12, c2=1e-12, a_star=1 - 1e-13)
        th[synth.I_A], th[synth.I_A + 1] = 1 - 1e-13, 1e-13
        p = H.problem(th, H=13, W=13, psfs=[H.psf_single(sig)] * 5, sky=150.0, seed=4)
        o = Oracle(p)
        _, g, _ = o.derivs(th[None])
        c1 = th[synth.I_C1:synth.I_C1 + 4]
        logl = [0.0] * 5
        logl[2] = th[synth.I_R1]
        logl[1] = logl[2] - c1[1]
        logl[0] = logl[1] - c1[0]
        logl[3] = logl[2] + c1[2]
        logl[4] = logl[3] + c1[3]
        iota = 1.0 / 0.005
        dll = 0.0
        for im in p.images:
            El = math.exp(logl[im.band])
            for row in range(13):
                for col in range(13):
                    gp = math.exp(-((col - ux) ** 2 + (row - uy) ** 2) / (2 * sig * sig)) / (2 * math.pi * sig * sig)
                    F = 150.0 + iota * El * gp
                    dll += (float(im.pixels[row, col]) / F - 1.0) * iota * El * gp
        mean_p, var_p = p.prior_r[0][0], p.prior_r[0][1]
        dkl = th[synth.I_A] * (th[synth.I_R1] - mean_p) / var_p
        want = dll - dkl
        assert abs(g[0, synth.I_R1] - want) <= 1e-8 * max(1.0, abs(dll))
