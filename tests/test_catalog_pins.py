"""Pins of the oracle's catalog rows and Table II error summary: the magnitude
convention, log-normal moments by Gauss-Hermite quadrature, per-band brightness
against the oracle's (separately pinned) brightness moments, the type mixture by
quadrature, the angle's period, and hand-worked error summaries."""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from oracle import catalog as OC
from oracle.oracle import brightness
from paper_1801_10277_gb300 import synth
from tests import helpers as H

COL = {f: i for i, f in enumerate(OC.FIELDS)}


def gh(n):
    x, w = hermegauss(n)
    return x, w / math.sqrt(2 * math.pi)


def random_theta(rng):
    th = H.star_theta(rng.uniform(0, 50), rng.uniform(0, 50))
    for i in range(2):
        th[synth.I_R1 + i] = rng.normal(1.0, 1.0)
        th[synth.I_R2 + i] = rng.uniform(0.001, 0.3)
        th[synth.I_C1 + 4 * i:synth.I_C1 + 4 * i + 4] = rng.normal(0, 0.5, 4)
        th[synth.I_C2 + 4 * i:synth.I_C2 + 4 * i + 4] = rng.uniform(0.001, 0.1, 4)
    a = rng.uniform(0.01, 0.99)
    th[synth.I_A:synth.I_A + 2] = [a, 1 - a]
    th[synth.I_ANGLE] = rng.uniform(-7, 7)
    return th


def test_field_layout_matches_header():
    from paper_1801_10277_gb300 import celeste
    assert OC.FIELDS == celeste.CAT_FIELDS and len(OC.FIELDS) == 54
    assert OC.SCORE_FIELDS == celeste.SCORE_FIELDS
    src = open(__file__.replace("tests/test_catalog_pins.py", "include/celeste.h")).read()
    for name, idx in (("CELESTE_CAT_GAL = 26", COL["gal_rmag"]), ("CELESTE_CAT_RFLUX_MIX = 48", COL["rflux_mix"]),
                      ("CELESTE_CAT_ANGLE_DEG = 52", COL["angle_deg"]),
                      ("CELESTE_CAT_STAR = 4", COL["star_rmag"])):
        assert name in src and int(name.split("= ")[1]) == idx
    assert COL["star_mag_u_sd"] == 4 + 17 and COL["gal_color_ug"] == 26 + 4


def test_magnitude_zero_point():
    # 1 nanomaggy is magnitude 22.5; a factor 100 in flux is 5 magnitudes
    th = H.star_theta(0, 0)
    th[synth.I_R1] = 0.0
    th[synth.I_R1 + 1] = math.log(100.0)
    row = OC.catalog_row(th)
    assert row[COL["star_rmag"]] == pytest.approx(22.5, abs=1e-14)
    assert row[COL["gal_rmag"]] == pytest.approx(17.5, abs=1e-13)


def test_lognormal_flux_moments_by_quadrature():
    x, w = gh(80)
    rng = np.random.default_rng(1)
    for _ in range(5):
        th = random_theta(rng)
        row = OC.catalog_row(th)
        for t, name in ((0, "star"), (1, "gal")):
            r1, r2 = th[synth.I_R1 + t], th[synth.I_R2 + t]
            l = np.exp(r1 + math.sqrt(r2) * x)
            m = w @ l
            sd = math.sqrt(w @ (l - m) ** 2)
            assert row[COL[f"{name}_rflux"]] == pytest.approx(m, rel=1e-12)
            assert row[COL[f"{name}_rflux_sd"]] == pytest.approx(sd, rel=1e-10)
            # the magnitude is Gaussian: its mean and sd by the same rule
            mag = 22.5 - 2.5 * np.log10(l)
            assert row[COL[f"{name}_rmag"]] == pytest.approx(w @ mag, rel=1e-13)
            assert row[COL[f"{name}_rmag_sd"]] == pytest.approx(math.sqrt(w @ (mag - w @ mag) ** 2), rel=1e-10)


def test_band_magnitudes_against_brightness_moments():
    """E[l_b | t] and E[l_b^2 | t] from the oracle's brightness code (pinned by a 5-D
    Gauss-Hermite rule over the colour definition) fix each band's log-normal
    parameters: v = log(E[l^2] / E[l]^2), mu = log E[l] - v / 2."""
    rng = np.random.default_rng(2)
    for _ in range(4):
        th = random_theta(rng)
        row = OC.catalog_row(th)
        k = 2.5 / math.log(10)
        for t, name in ((0, "star"), (1, "gal")):
            mus = []
            for b, band in enumerate("ugriz"):
                El, El2 = brightness(th, b, t)
                v = math.log(El2 / El ** 2)
                mu = math.log(El) - v / 2
                mus.append(mu)
                assert row[COL[f"{name}_mag_{band}"]] == pytest.approx(22.5 - k * mu, abs=1e-10)
                assert row[COL[f"{name}_mag_{band}_sd"]] == pytest.approx(k * math.sqrt(v), rel=1e-8)
            for j, c in enumerate(OC.COLOURS):   # colour = m_j - m_{j+1}
                assert row[COL[f"{name}_color_{c}"]] == pytest.approx(k * (mus[j + 1] - mus[j]), abs=1e-10)


def test_type_mixture_by_quadrature():
    x, w = gh(80)
    th = random_theta(np.random.default_rng(3))
    row = OC.catalog_row(th)
    a = th[synth.I_A:synth.I_A + 2]
    m1 = m2 = 0.0
    for t in range(2):
        l = np.exp(th[synth.I_R1 + t] + math.sqrt(th[synth.I_R2 + t]) * x)
        m1 += a[t] * (w @ l)
        m2 += a[t] * (w @ l ** 2)
    assert row[COL["rflux_mix"]] == pytest.approx(m1, rel=1e-12)
    assert row[COL["rflux_mix_sd"]] == pytest.approx(math.sqrt(m2 - m1 ** 2), rel=1e-8)


@pytest.mark.parametrize("phi,deg", [(0.0, 0.0), (-0.1, 180 - math.degrees(0.1)),
                                     (math.pi + 0.2, math.degrees(0.2)), (2.5, math.degrees(2.5)),
                                     (-3 * math.pi + 1.0, math.degrees(1.0))])
def test_angle_period(phi, deg):
    th = H.star_theta(0, 0)
    th[synth.I_ANGLE] = phi
    assert OC.catalog_row(th)[COL["angle_deg"]] == pytest.approx(deg, abs=1e-11)


def test_type_threshold():
    th = H.star_theta(0, 0)
    for a, s in ((0.5, 1.0), (0.4999999, 0.0), (0.9, 1.0)):
        th[synth.I_A:synth.I_A + 2] = [a, 1 - a]
        assert OC.catalog_row(th)[COL["is_star"]] == s


def _cat(rows):
    """Catalog rows from a few named fields (zeros elsewhere)."""
    out = np.zeros((len(rows), len(OC.FIELDS)))
    for i, r in enumerate(rows):
        for k, v in r.items():
            out[i, COL[k]] = v
    return out


def test_score_hand_worked():
    tru = _cat([dict(u0=0, u1=0, is_star=1, star_rmag=20, star_color_ug=1.0),
                dict(u0=10, u1=10, is_star=0, gal_rmag=19, gal_color_gr=0.5, e_dev=0.2, e_axis=0.5,
                     scale=2.0, angle_deg=1.0),
                dict(u0=5, u1=5, is_star=0, gal_rmag=18, e_dev=0.7, e_axis=0.9, scale=3.0, angle_deg=90.0)])
    est = _cat([dict(u0=3, u1=4, is_star=0, gal_rmag=20.5, gal_color_ug=0.25),      # star called galaxy
                dict(u0=10, u1=10, is_star=0, gal_rmag=19.2, gal_color_gr=0.3, e_dev=0.3, e_axis=0.4,
                     scale=2.5, angle_deg=179.0),
                dict(u0=5, u1=6, is_star=1, star_rmag=18.0, e_dev=0.7, e_axis=0.9, scale=3.0,
                     angle_deg=100.0)])                                             # galaxy called star
    s = OC.score(est, tru)
    assert s["position"] == pytest.approx((5 + 0 + 1) / 3)
    assert s["brightness"] == pytest.approx((0.5 + 0.2 + 0.0) / 3)
    assert s["color_ug"] == pytest.approx(0.75 / 3)
    assert s["color_gr"] == pytest.approx(0.2 / 3)
    assert s["missed_star"] == 1.0 and s["missed_gal"] == 0.5
    assert s["n_gal"] == 2 and s["n_star"] == 1
    assert s["profile"] == pytest.approx(0.05) and s["axis"] == pytest.approx(0.05)
    assert s["scale"] == pytest.approx(0.25)
    assert s["angle_deg"] == pytest.approx((2.0 + 10.0) / 2)   # 179 vs 1 degree is 2 degrees


def test_score_degenerate_cases():
    empty = np.zeros((0, len(OC.FIELDS)))
    assert all(v == 0.0 for v in OC.score(empty, empty).values())
    stars = _cat([dict(is_star=1, star_rmag=20)] * 3)
    s = OC.score(stars, stars)
    assert s["n_gal"] == 0 and s["missed_gal"] == 0 and s["profile"] == 0
    assert all(v == 0.0 for k, v in s.items() if k != "n_star") and s["n_star"] == 3
