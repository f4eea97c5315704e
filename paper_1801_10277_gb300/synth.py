"""Seeded synthetic SDSS-shaped inputs: images, PSFs, priors, variational starts,
patches and neighbour lists.

This module only draws inputs.  It holds none of the method's arithmetic: pixel
counts are Poisson draws around a sky level plus one isotropic Gaussian blob per
source (a stand-in for real sky, not the model's PSF x profile mixture), and the
patch rule uses the same blob.  Both the CPU oracle and the CUDA path consume
exactly the arrays made here.

Parameter layout of one source (44 doubles, constrained coordinates; Section III
names the quantities, Section IV gives the count of 44)::

    0,1    u        position (world coords; pixel coords of image 0 for one field)
    2      e_dev    de Vaucouleurs proportion of the galaxy profile
    3      e_axis   minor / major axis ratio
    4      e_angle  major-axis angle, radians, counter-clockwise from +x (column)
    5      e_scale  half-light radius along the major axis, pixels
    6,7    r1[i]    mean of log reference-band (r) brightness given type i
    8,9    r2[i]    variance of log brightness given type i
    10..17 c1[i][j] colour means, index 10 + 4 i + j (j: u-g, g-r, r-i, i-z)
    18..25 c2[i][j] colour variances, index 18 + 4 i + j
    26,27  a[i]     P(star), P(galaxy)
    28..43 k[i][d]  colour-prior component responsibilities, index 28 + 8 i + d

Type i = 0 is a star, i = 1 a galaxy.  Bands are u, g, r, i, z (0..4).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

NPARAM = 44
NBANDS = 5
REF_BAND = 2
NCOLOR = 4
NPRIOR_COMP = 8

I_U, I_EDEV, I_AXIS, I_ANGLE, I_SCALE = 0, 2, 3, 4, 5
I_R1, I_R2, I_C1, I_C2, I_A, I_K = 6, 8, 10, 18, 26, 28

_HERE = os.path.dirname(os.path.abspath(__file__))


def load_profiles():
    with open(os.path.join(_HERE, "data", "profiles.json")) as f:
        d = json.load(f)
    return np.array(d["exp"], dtype=np.float64), np.array(d["dev"], dtype=np.float64)


@dataclass
class Image:
    band: int
    pixels: np.ndarray            # [H][W] float32 counts
    sky: float                    # counts per pixel
    calib: float                  # nanomaggies per count (iota = 1 / calib)
    wcs: np.ndarray               # [6]: A00 A01 A10 A11 t0 t1; pixel = A u + t
    psf: np.ndarray               # [K][6]: alpha, xi_x, xi_y, Sxx, Sxy, Syy
    sky_map: np.ndarray | None = None   # optional [H][W] float32 sky counts
    # optional smooth distortion added to the affine map (a stand-in for a sky survey's WCS):
    # (cx, cy, L, d1, d2, d3, d4), pixel = A u + t + (d1 x^2 + d2 x y, d3 y^2 + d4 x y)
    # with x = (u0 - cx) / L, y = (u1 - cy) / L
    warp: tuple | None = None

    @property
    def height(self):
        return self.pixels.shape[0]

    @property
    def width(self):
        return self.pixels.shape[1]


@dataclass
class Problem:
    images: list
    exp_mix: np.ndarray           # [Je][2] weight, variance
    dev_mix: np.ndarray           # [Jd][2]
    prior_star: float
    prior_r: np.ndarray           # [2][2]: mean, variance of log r per type
    prior_c: np.ndarray           # [2][D][21]: weight, mean[4], cov[4][4]
    theta: np.ndarray             # [S][44] starting variational parameters
    truth: np.ndarray             # [S][44] parameters the blobs were drawn from
    patch_offsets: np.ndarray     # [S+1] int32
    patches: np.ndarray           # [P][5] int32: image, x0, y0, w, h
    nbr_offsets: np.ndarray       # [S+1] int32
    nbrs: np.ndarray              # [E] int32
    name: str = ""
    meta: dict = field(default_factory=dict)
    patch_wcs: np.ndarray | None = None   # optional [P][6]: each patch's map, linearised at its source

    @property
    def n_src(self):
        return self.theta.shape[0]

    def source_pixels(self):
        """Number of (source, active pixel) pairs over all patches."""
        return int(np.sum(self.patches[:, 3].astype(np.int64) * self.patches[:, 4]))


# ----------------------------------------------------------------------------------
# draws


def _rot(phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, -s], [s, c]])


def draw_psf(rng, sigma_lo=1.0, sigma_hi=2.5, k=3):
    w = np.sort(rng.dirichlet([5.0, 3.0, 2.0][:k]))[::-1]
    sig = np.sort(rng.uniform(sigma_lo, sigma_hi, size=k))
    out = np.zeros((k, 6))
    for j in range(k):
        e = rng.uniform(0.85, 1.0)
        R = _rot(rng.uniform(0, math.pi))
        S = sig[j] ** 2 * R @ np.diag([1.0, e * e]) @ R.T
        out[j] = [w[j], rng.normal(0, 0.05), rng.normal(0, 0.05), S[0, 0], S[0, 1], S[1, 1]]
    return out


def draw_priors(rng, D=NPRIOR_COMP):
    prior_r = np.array([[math.log(5.0), 1.2 ** 2], [math.log(5.0), 1.2 ** 2]])
    prior_c = np.zeros((2, D, 21))
    for i in range(2):
        for d in range(D):
            prior_c[i, d, 0] = 1.0 / D
            prior_c[i, d, 1:5] = rng.normal(0, 0.5, size=4)
            prior_c[i, d, 5:] = (0.25 * np.eye(4)).ravel()
    return 0.4, prior_r, prior_c


def band_log_flux(log_r, colors):
    """log brightness per band from the reference-band log brightness and the four
    adjacent-band log ratios (Section III: colours are log ratios of adjacent bands)."""
    c = colors
    return np.array([log_r - c[0] - c[1], log_r - c[1], log_r, log_r + c[2], log_r + c[2] + c[3]])


def draw_truth(rng, n, gal_frac=0.6, bright_frac=0.0):
    t = np.zeros((n, NPARAM))
    is_gal = rng.uniform(size=n) < gal_frac
    flux = np.exp(rng.normal(math.log(5.0), 1.2, size=n))
    if bright_frac > 0:
        b = rng.uniform(size=n) < bright_frac
        flux[b] = rng.uniform(500.0, 5000.0, size=b.sum())
    colors = rng.normal(0, 0.5, size=(n, 4))
    t[:, I_EDEV] = rng.uniform(0.05, 0.95, size=n)
    t[:, I_AXIS] = rng.uniform(0.2, 1.0, size=n)
    t[:, I_ANGLE] = rng.uniform(0, math.pi, size=n)
    t[:, I_SCALE] = np.exp(rng.normal(math.log(2.0), 0.6, size=n))
    for i in range(2):
        t[:, I_R1 + i] = np.log(flux)
        t[:, I_R2 + i] = 1e-4
        t[:, I_C1 + 4 * i:I_C1 + 4 * i + 4] = colors
        t[:, I_C2 + 4 * i:I_C2 + 4 * i + 4] = 1e-4
        t[:, I_K + 8 * i:I_K + 8 * i + 8] = 1.0 / 8
    t[:, I_A] = np.where(is_gal, 0.0, 1.0)
    t[:, I_A + 1] = 1.0 - t[:, I_A]
    return t, is_gal


def perturb_start(rng, truth, is_gal, pos_jit=0.5, flux_jit=0.2):
    th = truth.copy()
    n = th.shape[0]
    th[:, 0:2] += rng.uniform(-pos_jit, pos_jit, size=(n, 2))
    f = rng.uniform(1 - flux_jit, 1 + flux_jit, size=n)
    for i in range(2):
        th[:, I_R1 + i] = truth[:, I_R1 + i] + np.log(f)
        th[:, I_R2 + i] = 0.05
        th[:, I_C1 + 4 * i:I_C1 + 4 * i + 4] += rng.normal(0, 0.1, size=(n, 4))
        th[:, I_C2 + 4 * i:I_C2 + 4 * i + 4] = 0.02
    th[:, I_A] = np.where(is_gal, 0.3, 0.7)
    th[:, I_A + 1] = 1.0 - th[:, I_A]
    star = ~is_gal
    th[star, I_EDEV] = 0.5
    th[star, I_AXIS] = 0.8
    th[star, I_ANGLE] = 0.3
    th[star, I_SCALE] = 1.0
    gal = is_gal
    th[gal, I_EDEV] = np.clip(th[gal, I_EDEV] + rng.normal(0, 0.05, size=gal.sum()), 0.05, 0.95)
    th[gal, I_AXIS] = np.clip(th[gal, I_AXIS] * rng.uniform(0.9, 1.1, size=gal.sum()), 0.1, 0.95)
    th[gal, I_ANGLE] += rng.normal(0, 0.1, size=gal.sum())
    th[gal, I_SCALE] *= rng.uniform(0.85, 1.15, size=gal.sum())
    return th


# ----------------------------------------------------------------------------------
# blob images and patches (input synthesis only; not the model)


def _psf_var(psf):
    return float(np.sum(psf[:, 0] * 0.5 * (psf[:, 3] + psf[:, 5])))


def _blob_var(psf, is_gal, scale, widen=1.5):
    return _psf_var(psf) + (float((widen * scale) ** 2) if is_gal else 0.0)


def pixel_position(wcs, u):
    A = np.array(wcs[:4]).reshape(2, 2)
    return A @ np.asarray(u) + np.array(wcs[4:6])


def pixel_position_full(im, u):
    """The image's full world -> pixel map (affine part plus its distortion)."""
    p = pixel_position(im.wcs, u)
    if im.warp is not None:
        cx, cy, L, d1, d2, d3, d4 = im.warp
        x, y = (u[0] - cx) / L, (u[1] - cy) / L
        p = p + np.array([d1 * x * x + d2 * x * y, d3 * y * y + d4 * x * y])
    return p


def linearised_wcs(im, u0):
    """The image's map linearised at u0: pixel ~ J (u - u0) + p(u0) = J u + t, in the
    wcs layout (J00 J01 J10 J11 t0 t1)."""
    J = np.array(im.wcs[:4], np.float64).reshape(2, 2).copy()
    if im.warp is not None:
        cx, cy, L, d1, d2, d3, d4 = im.warp
        x, y = (u0[0] - cx) / L, (u0[1] - cy) / L
        J += np.array([[2 * d1 * x + d2 * y, d2 * x], [d4 * y, 2 * d3 * y + d4 * x]]) / L
    t = pixel_position_full(im, u0) - J @ np.asarray(u0, np.float64)
    return np.array([J[0, 0], J[0, 1], J[1, 0], J[1, 1], t[0], t[1]])


def render_blobs(rng, images, truth, is_gal):
    """Poisson counts: sky + one isotropic Gaussian blob per (source, image)."""
    for im in images:
        H, W = im.height, im.width
        rate = np.full((H, W), im.sky, dtype=np.float64)
        iota = 1.0 / im.calib
        for s in range(truth.shape[0]):
            lf = band_log_flux(truth[s, I_R1], truth[s, I_C1:I_C1 + 4])[im.band]
            cnt = iota * math.exp(lf)
            v = _blob_var(im.psf, bool(is_gal[s]), truth[s, I_SCALE])
            px, py = pixel_position_full(im, truth[s, 0:2])
            rad = int(math.ceil(5 * math.sqrt(v)))
            x0, x1 = max(0, int(px) - rad), min(W, int(px) + rad + 1)
            y0, y1 = max(0, int(py) - rad), min(H, int(py) + rad + 1)
            if x0 >= x1 or y0 >= y1:
                continue
            xs = np.arange(x0, x1) - px
            ys = np.arange(y0, y1) - py
            gx = np.exp(-xs ** 2 / (2 * v))
            gy = np.exp(-ys ** 2 / (2 * v))
            rate[y0:y1, x0:x1] += cnt / (2 * math.pi * v) * np.outer(gy, gx)
        im.pixels = rng.poisson(rate).astype(np.float32)


def patch_width(im, theta_s, is_gal_s):
    """Odd square patch side from the reference-band blob: the radius where the blob
    falls below 0.1 sqrt(sky), side 2 ceil(R) + 1 clamped to [15, 101]."""
    lf = float(theta_s[I_R1])
    cnt = math.exp(lf) / im.calib
    # galaxies get a wider envelope than the rendered blob: the de Vaucouleurs
    # profile keeps light far beyond its half-light radius
    v = _blob_var(im.psf, is_gal_s, float(theta_s[I_SCALE]), widen=3.0)
    peak = cnt / (2 * math.pi * v)
    thr = 0.1 * math.sqrt(im.sky)
    R = math.sqrt(2 * v * math.log(peak / thr)) if peak > thr else 0.0
    return int(min(101, max(15, 2 * math.ceil(R) + 1)))


def make_patches(images, theta, is_gal):
    ref = next(i for i, im in enumerate(images) if im.band == REF_BAND)
    offs = [0]
    rows = []
    for s in range(theta.shape[0]):
        w = patch_width(images[ref], theta[s], bool(is_gal[s]))
        for n, im in enumerate(images):
            px, py = pixel_position_full(im, theta[s, 0:2])
            cx, cy = int(round(px)), int(round(py))
            x0, y0 = cx - w // 2, cy - w // 2
            x1, y1 = x0 + w, y0 + w
            x0c, y0c = max(0, x0), max(0, y0)
            x1c, y1c = min(im.width, x1), min(im.height, y1)
            if x1c <= x0c or y1c <= y0c:
                continue
            rows.append((n, x0c, y0c, x1c - x0c, y1c - y0c))
        offs.append(len(rows))
    return np.array(offs, dtype=np.int32), np.array(rows, dtype=np.int32).reshape(-1, 5)


def make_neighbours(n_src, patch_offsets, patches, cell=128):
    """Sources are neighbours when their patches intersect in some image."""
    owner = np.repeat(np.arange(n_src), np.diff(patch_offsets))
    nb = [set() for _ in range(n_src)]
    grid = {}
    for p in range(patches.shape[0]):
        n, x0, y0, w, h = (int(v) for v in patches[p])
        for cx in range(x0 // cell, (x0 + w - 1) // cell + 1):
            for cy in range(y0 // cell, (y0 + h - 1) // cell + 1):
                grid.setdefault((n, cx, cy), []).append(p)
    for lst in grid.values():
        for a_i in range(len(lst)):
            pa = patches[lst[a_i]]
            for b_i in range(a_i + 1, len(lst)):
                pb = patches[lst[b_i]]
                if (pa[1] < pb[1] + pb[3] and pb[1] < pa[1] + pa[3] and
                        pa[2] < pb[2] + pb[4] and pb[2] < pa[2] + pa[4]):
                    sa, sb = int(owner[lst[a_i]]), int(owner[lst[b_i]])
                    if sa != sb:
                        nb[sa].add(sb)
                        nb[sb].add(sa)
    offs = np.zeros(n_src + 1, dtype=np.int32)
    flat = []
    for s in range(n_src):
        lst = sorted(nb[s])
        flat.extend(lst)
        offs[s + 1] = len(flat)
    return offs, np.array(flat, dtype=np.int32)


# ----------------------------------------------------------------------------------
# the five workloads


def _single_field_images(rng, H, W, sky=150.0, calib=0.005, wcs=None):
    wcs = np.array([1, 0, 0, 1, 0, 0], dtype=np.float64) if wcs is None else wcs
    return [Image(band=b, pixels=np.zeros((H, W), np.float32), sky=sky, calib=calib,
                  wcs=wcs.copy(), psf=draw_psf(rng)) for b in range(NBANDS)]


def _finish(rng, name, images, truth, is_gal, theta, meta=None):
    exp_mix, dev_mix = load_profiles()
    prior_star, prior_r, prior_c = draw_priors(rng)
    render_blobs(rng, images, truth, is_gal)
    po, pa = make_patches(images, theta, is_gal)
    no, nb = make_neighbours(truth.shape[0], po, pa)
    pw = None
    if any(im.warp is not None for im in images):
        # each patch's map linearised at its source's starting (catalog) position
        owner = np.repeat(np.arange(truth.shape[0]), np.diff(po))
        pw = np.stack([linearised_wcs(images[int(pa[p, 0])], theta[owner[p], 0:2])
                       for p in range(pa.shape[0])]) if len(pa) else np.zeros((0, 6))
    return Problem(images=images, exp_mix=exp_mix, dev_mix=dev_mix, prior_star=prior_star,
                   prior_r=prior_r, prior_c=prior_c, theta=theta, truth=truth,
                   patch_offsets=po, patches=pa, nbr_offsets=no, nbrs=nb, name=name,
                   meta=meta or {}, patch_wcs=pw)


def tiny_two_source(seed=2026, H=48, W=48):
    """Two overlapping sources (a star and a galaxy with e_dev 0.3, axis ratio 0.6,
    angle 40 degrees, half-light radius 2 px) in five 48 x 48 band images."""
    rng = np.random.default_rng(seed)
    images = _single_field_images(rng, H, W)
    truth, _ = draw_truth(rng, 2)
    is_gal = np.array([False, True])
    truth[0, 0:2] = [W * 0.45, H * 0.5]
    truth[1, 0:2] = [W * 0.58, H * 0.52]
    truth[1, I_EDEV], truth[1, I_AXIS] = 0.3, 0.6
    truth[1, I_ANGLE], truth[1, I_SCALE] = math.radians(40.0), 2.0
    for i in range(2):
        truth[:, I_R1 + i] = math.log(20.0)
    truth[:, I_A] = [1.0, 0.0]
    truth[:, I_A + 1] = [0.0, 1.0]
    theta = perturb_start(rng, truth, is_gal)
    return _finish(rng, "tiny_2src_5x48x48", images, truth, is_gal, theta)


def one_field(seed=2027, n_src=500, H=1489, W=2048, gal_frac=0.6, bright_frac=0.0):
    """One SDSS-shaped field: 5 bands of 2048 x 1489 px, uniform source positions."""
    rng = np.random.default_rng(seed)
    images = _single_field_images(rng, H, W)
    truth, is_gal = draw_truth(rng, n_src, gal_frac, bright_frac)
    truth[:, 0] = rng.uniform(0, W - 1, size=n_src)
    truth[:, 1] = rng.uniform(0, H - 1, size=n_src)
    theta = perturb_start(rng, truth, is_gal)
    return _finish(rng, f"field_{n_src}src_5x{W}x{H}", images, truth, is_gal, theta)


def crowded_region(seed=2028, n_src=64, H=256, W=256, lo=2, hi=12, max_rounds=400):
    """A 256 x 256 x 5 region whose 64 sources each have 2-12 neighbours: clustered
    placement, re-drawing any source whose neighbour count falls outside [lo, hi]."""
    rng = np.random.default_rng(seed)
    images = _single_field_images(rng, H, W)
    truth, is_gal = draw_truth(rng, n_src)
    n_cl = 6
    centres = rng.uniform(40, W - 40, size=(n_cl, 2))

    def place(idx):
        c = centres[rng.integers(n_cl, size=len(idx))]
        truth[idx, 0:2] = np.clip(c + rng.normal(0, 22, size=(len(idx), 2)), 2, W - 3)

    place(np.arange(n_src))
    for _ in range(max_rounds):
        theta = perturb_start(np.random.default_rng(seed + 1), truth, is_gal)
        po, pa = make_patches(images, theta, is_gal)
        no, _ = make_neighbours(n_src, po, pa)
        cnt = np.diff(no)
        bad = np.where((cnt < lo) | (cnt > hi))[0]
        if len(bad) == 0:
            break
        place(bad[:max(1, len(bad) // 2)])
    theta = perturb_start(np.random.default_rng(seed + 1), truth, is_gal)
    return _finish(rng, f"crowded_{n_src}src_5x{W}x{H}", images, truth, is_gal, theta)


def multi_epoch(seed=2029, n_src=20000, n_fields=8, H=1489, W=2048, stride=400):
    """Eight overlapping 2048 x 1489 fields offset along x by 400 px (each sky point
    covered 1-6 times), each with per-image PSF, sky U(100,200) and calibration
    U(0.004,0.006), and a small per-field affine distortion."""
    rng = np.random.default_rng(seed)
    images = []
    for f in range(n_fields):
        ang = rng.normal(0, 2e-3)
        sc = 1.0 + rng.normal(0, 1e-3)
        A = sc * _rot(ang)
        off = np.array([f * stride, rng.uniform(-40, 40)])
        # pixel = A (u - off)
        t = -A @ off
        wcs = np.array([A[0, 0], A[0, 1], A[1, 0], A[1, 1], t[0], t[1]])
        for b in range(NBANDS):
            images.append(Image(band=b, pixels=np.zeros((H, W), np.float32),
                                sky=rng.uniform(100, 200), calib=rng.uniform(0.004, 0.006),
                                wcs=wcs.copy(), psf=draw_psf(rng)))
    truth, is_gal = draw_truth(rng, n_src)
    truth[:, 0] = rng.uniform(0, (n_fields - 1) * stride + W - 1, size=n_src)
    truth[:, 1] = rng.uniform(0, H - 1, size=n_src)
    theta = perturb_start(rng, truth, is_gal)
    return _finish(rng, f"multiepoch_{n_src}src_{n_fields}x5x{W}x{H}", images, truth,
                   is_gal, theta)


def deep_stack(seed=2031, n_src=100, n_epochs=96, H=400, W=400, field_size=384):
    """A deeply imaged patch of sky (like the repeatedly scanned stripe): 96 epochs x 5
    bands = 480 images of 400 x 400 px, each with its own pointing offset (+-8 px),
    rotation (1e-2 rad), scale (3e-3), PSF, sky U(100, 200), calibration
    U(0.004, 0.006) and a smooth quadratic distortion of up to ~1 px; 100 sources, so
    every source has 480 patches, each with its image's map linearised at the source."""
    rng = np.random.default_rng(seed)
    images = []
    c = field_size / 2.0
    for e in range(n_epochs):
        A = (1.0 + rng.normal(0, 3e-3)) * _rot(rng.normal(0, 1e-2))
        off = np.array([W / 2.0, H / 2.0]) + rng.uniform(-8, 8, size=2)
        t = off - A @ np.array([c, c])           # the field centre lands near the image centre
        wcs = np.array([A[0, 0], A[0, 1], A[1, 0], A[1, 1], t[0], t[1]])
        warp = (c, c, c, *rng.normal(0, 0.3, size=4))
        for b in range(NBANDS):
            images.append(Image(band=b, pixels=np.zeros((H, W), np.float32),
                                sky=rng.uniform(100, 200), calib=rng.uniform(0.004, 0.006),
                                wcs=wcs.copy(), psf=draw_psf(rng), warp=warp))
    truth, is_gal = draw_truth(rng, n_src)
    truth[:, 0:2] = rng.uniform(12, field_size - 12, size=(n_src, 2))
    theta = perturb_start(rng, truth, is_gal)
    return _finish(rng, f"deepstack_{n_src}src_{n_epochs}x5x{W}x{H}", images, truth, is_gal, theta)


def config(idx, seed=None, **kw):
    """The workloads by index: 0 tiny two-source, 1 one field of 500 sources,
    2 crowded 64-source region, 3 multi-epoch 20k sources, 4 is built per field by
    ``many_fields`` (200k sources over 64 fields) and sampled, 5 deep stack (480
    images per source, distorted maps linearised per source), 6 the whole sweep (the
    64 fields of 4 as one 200,000-source problem)."""
    base = 2026 + idx if seed is None else seed
    if idx == 0:
        return tiny_two_source(base, **kw)
    if idx == 1:
        return one_field(base, **kw)
    if idx == 2:
        return crowded_region(base, **kw)
    if idx == 3:
        return multi_epoch(base, **kw)
    if idx == 4:
        return many_fields_sample(base, **kw)
    if idx == 5:
        return deep_stack(base, **kw)
    if idx == 6:
        return full_sweep(2030 if seed is None else seed, **kw)
    raise ValueError(idx)


def many_fields_sample(seed=2030, n_fields_sampled=1, n_src_per_field=3125, bright_frac=0.1):
    """One of the 64 fields of the 200,000-source sweep (3125 sources per field,
    10 % bright with flux U(500, 5000) nmgy).  Fields are disjoint, so a field is an
    independent unit of the sweep."""
    out = one_field(seed, n_src=n_src_per_field * n_fields_sampled, bright_frac=bright_frac)
    out.name = f"sweep_field_{out.n_src}src_bright{bright_frac}"
    return out


def full_sweep(seed=2030, n_fields=64, n_src_per_field=3125, bright_frac=0.1, gap=52):
    """The whole 200,000-source sweep as one problem: 64 disjoint fields (field f drawn
    as the sweep field with seed + 7919 f, so field 0 is the sampled sweep field), laid
    side by side in one world frame 2048 + gap px apart along x; each field's images map
    their own strip (pixel = u - (f (2048 + gap), 0))."""
    fields = [one_field(seed + 7919 * f, n_src=n_src_per_field, bright_frac=bright_frac)
              for f in range(n_fields)]
    images, thetas, truths, po, pa, no, nb = [], [], [], [0], [], [0], []
    n0 = 0
    for f, fld in enumerate(fields):
        dx = f * (fld.images[0].width + gap)
        for im in fld.images:
            im.wcs = im.wcs.copy()
            im.wcs[4] -= dx
            images.append(im)
        th, tr = fld.theta.copy(), fld.truth.copy()
        th[:, 0] += dx
        tr[:, 0] += dx
        thetas.append(th)
        truths.append(tr)
        rows = fld.patches.copy()
        rows[:, 0] += NBANDS * f
        pa.append(rows)
        po.extend((fld.patch_offsets[1:] + po[-1]).tolist())
        nb.append(fld.nbrs + n0)
        no.extend((fld.nbr_offsets[1:] + no[-1]).tolist())
        n0 += fld.n_src
    f0 = fields[0]
    return Problem(images=images, exp_mix=f0.exp_mix, dev_mix=f0.dev_mix, prior_star=f0.prior_star,
                   prior_r=f0.prior_r, prior_c=f0.prior_c, theta=np.concatenate(thetas),
                   truth=np.concatenate(truths), patch_offsets=np.array(po, np.int32),
                   patches=np.concatenate(pa).astype(np.int32), nbr_offsets=np.array(no, np.int32),
                   nbrs=np.concatenate(nb).astype(np.int32),
                   name=f"sweep_{n0}src_{n_fields}x5x{f0.images[0].width}x{f0.images[0].height}")


def subset(prob, idx):
    """The sub-problem made of sources `idx` (ascending), their patches and the
    neighbour relations among them; images and priors are shared."""
    idx = np.asarray(sorted(int(i) for i in idx))
    remap = -np.ones(prob.n_src, dtype=np.int64)
    remap[idx] = np.arange(len(idx))
    offs = [0]
    rows = []
    nb_off = [0]
    nb = []
    keep_p = []
    for s in idx:
        rows.extend(prob.patches[prob.patch_offsets[s]:prob.patch_offsets[s + 1]].tolist())
        keep_p.extend(range(prob.patch_offsets[s], prob.patch_offsets[s + 1]))
        offs.append(len(rows))
        for o in prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]]:
            if remap[o] >= 0:
                nb.append(int(remap[o]))
        nb_off.append(len(nb))
    return Problem(images=prob.images, exp_mix=prob.exp_mix, dev_mix=prob.dev_mix,
                   prior_star=prob.prior_star, prior_r=prob.prior_r, prior_c=prob.prior_c,
                   theta=prob.theta[idx].copy(), truth=prob.truth[idx].copy(),
                   patch_offsets=np.array(offs, np.int32),
                   patches=np.array(rows, np.int32).reshape(-1, 5),
                   nbr_offsets=np.array(nb_off, np.int32), nbrs=np.array(nb, np.int32),
                   name=f"{prob.name}_subset{len(idx)}", meta=dict(prob.meta),
                   patch_wcs=None if prob.patch_wcs is None else prob.patch_wcs[keep_p].copy())
