"""Catalog rows with posterior uncertainty and the Table II error summary, written out
in plain FP64 numpy from their definitions.

TEST INFRASTRUCTURE ONLY: tests and the smoke check compare the library's catalog and
score entry points with these functions.

Definitions (Section III model; Section VIII for what a catalog reports):
* type: q(star) = a_star; the classified type is star when a_star >= 1/2;
* given type t, log l_r ~ N(r1_t, r2_t) and the four colours c_j = log(l_{j+1} / l_j)
  over u g r i z are independent N(c1_tj, c2_tj); each band's log flux is the r-band
  log flux plus or minus the colours between r and that band, so it is Gaussian;
* magnitudes use the nanomaggy zero point: m = 22.5 - 2.5 log10(l / nmgy);
* a log-normal flux with log-mean mu and log-variance v has mean exp(mu + v / 2) and
  standard deviation mean * sqrt(exp(v) - 1);
* the type-marginal flux is the two-component mixture over types with weights
  a_star + a_gal = 1.
"""
from __future__ import annotations

import numpy as np

NP = 44
U, EDEV, AXIS, ANGLE, SCALE, R1, R2, C1, C2, A = 0, 2, 3, 4, 5, 6, 8, 10, 18, 26

COLOURS = ("ug", "gr", "ri", "iz")
TYPE_FIELDS = (["rmag", "rmag_sd", "rflux", "rflux_sd"] + [f"color_{c}" for c in COLOURS]
               + [f"color_{c}_sd" for c in COLOURS] + [f"mag_{b}" for b in "ugriz"]
               + [f"mag_{b}_sd" for b in "ugriz"])
FIELDS = (["u0", "u1", "p_star", "is_star"] + [f"star_{f}" for f in TYPE_FIELDS]
          + [f"gal_{f}" for f in TYPE_FIELDS]
          + ["rflux_mix", "rflux_mix_sd", "e_dev", "e_axis", "angle_deg", "scale"])
SCORE_FIELDS = ["position", "missed_gal", "missed_star", "brightness"] + \
    [f"color_{c}" for c in COLOURS] + ["profile", "axis", "scale", "angle_deg", "n_gal", "n_star"]


def magnitude(log_flux):
    """m = 22.5 - 2.5 log10(l), l in nanomaggies."""
    return 22.5 - 2.5 * np.asarray(log_flux) / np.log(10.0)


def band_log_moments(r1, r2, c1, c2):
    """Mean and variance of log l_b for b = u g r i z, walking outward from the r band:
    l_g = l_r / exp(c_gr), l_u = l_g / exp(c_ug), l_i = l_r exp(c_ri), l_z = l_i exp(c_iz)."""
    ug, gr, ri, iz = c1
    vug, vgr, vri, viz = c2
    mean = [r1 - gr - ug, r1 - gr, r1, r1 + ri, r1 + ri + iz]
    var = [r2 + vgr + vug, r2 + vgr, r2, r2 + vri, r2 + vri + viz]
    return np.array(mean), np.array(var)


def lognormal_mean_sd(mu, v):
    mean = np.exp(mu + v / 2.0)
    return mean, mean * np.sqrt(np.expm1(v))


def catalog_row(th):
    th = np.asarray(th, np.float64)
    row = {"u0": th[U], "u1": th[U + 1], "p_star": th[A], "is_star": 1.0 if th[A] >= 0.5 else 0.0}
    k = 2.5 / np.log(10.0)   # magnitudes per unit of natural log flux
    means, sds = [], []
    for t, name in ((0, "star"), (1, "gal")):
        r1, r2 = th[R1 + t], th[R2 + t]
        c1, c2 = th[C1 + 4 * t:C1 + 4 * t + 4], th[C2 + 4 * t:C2 + 4 * t + 4]
        row[f"{name}_rmag"] = magnitude(r1)
        row[f"{name}_rmag_sd"] = k * np.sqrt(r2)
        m, sd = lognormal_mean_sd(r1, r2)
        row[f"{name}_rflux"], row[f"{name}_rflux_sd"] = m, sd
        means.append(m)
        sds.append(sd)
        for j, c in enumerate(COLOURS):
            # m_j - m_{j+1} = -2.5 log10(l_j / l_{j+1}) = (2.5 / ln 10) c_j
            row[f"{name}_color_{c}"] = k * c1[j]
            row[f"{name}_color_{c}_sd"] = k * np.sqrt(c2[j])
        bm, bv = band_log_moments(r1, r2, c1, c2)
        for b, band in enumerate("ugriz"):
            row[f"{name}_mag_{band}"] = magnitude(bm[b])
            row[f"{name}_mag_{band}_sd"] = k * np.sqrt(bv[b])
    a = th[A:A + 2]
    mix = a[0] * means[0] + a[1] * means[1]
    # law of total variance: E[Var(l | t)] + Var(E[l | t])
    var = sum(a[t] * sds[t] ** 2 for t in range(2)) + sum(a[t] * (means[t] - mix) ** 2 for t in range(2))
    row["rflux_mix"] = mix
    row["rflux_mix_sd"] = np.sqrt(var)
    row["e_dev"], row["e_axis"], row["scale"] = th[EDEV], th[AXIS], th[SCALE]
    row["angle_deg"] = np.degrees(np.mod(th[ANGLE], np.pi)) % 180.0   # period pi
    return np.array([row[f] for f in FIELDS], np.float64)


def catalog(theta):
    theta = np.asarray(theta, np.float64).reshape(-1, NP)
    return np.stack([catalog_row(t) for t in theta]) if len(theta) else np.zeros((0, len(FIELDS)))


def score(est, tru):
    """Table II: mean errors of an estimated catalog against the truth.  Brightness and
    colours of each catalog come from its own classified type; the galaxy shape errors,
    and the share of galaxies called stars, are over the true galaxies; the share of
    stars called galaxies over the true stars.  Means over an empty set are 0."""
    col = {f: i for i, f in enumerate(FIELDS)}
    est = np.asarray(est, np.float64)
    tru = np.asarray(tru, np.float64)
    n = est.shape[0]
    out = dict.fromkeys(SCORE_FIELDS, 0.0)
    if n == 0:
        return out

    def typed(cat, field):
        star = cat[:, col["is_star"]] != 0
        return np.where(star, cat[:, col[f"star_{field}"]], cat[:, col[f"gal_{field}"]])

    d = np.hypot(est[:, col["u0"]] - tru[:, col["u0"]], est[:, col["u1"]] - tru[:, col["u1"]])
    out["position"] = d.mean()
    out["brightness"] = np.abs(typed(est, "rmag") - typed(tru, "rmag")).mean()
    for c in COLOURS:
        out[f"color_{c}"] = np.abs(typed(est, f"color_{c}") - typed(tru, f"color_{c}")).mean()
    t_star = tru[:, col["is_star"]] != 0
    e_star = est[:, col["is_star"]] != 0
    gal = ~t_star
    out["n_gal"], out["n_star"] = float(gal.sum()), float(t_star.sum())
    if gal.any():
        out["missed_gal"] = e_star[gal].mean()
        for f, key in (("e_dev", "profile"), ("e_axis", "axis"), ("scale", "scale")):
            out[key] = np.abs(est[gal, col[f]] - tru[gal, col[f]]).mean()
        da = np.abs(est[gal, col["angle_deg"]] - tru[gal, col["angle_deg"]])
        out["angle_deg"] = np.minimum(da, 180.0 - da).mean()
    if t_star.any():
        out["missed_star"] = (~e_star[t_star]).mean()
    return {k: float(v) for k, v in out.items()}
