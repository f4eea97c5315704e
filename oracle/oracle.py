"""ctypes binding of the FP64 C++ oracle (``celeste_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU-baseline leg
use it to produce expected values.  ``build()`` compiles the oracle with g++ (no
fast-math, no FMA contraction) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "celeste_oracle.cpp")
LIB = os.path.join(HERE, "_build", "liboracle.so")
NP_ = 44
NT_ = 41

_lib = None


def build(force=False):
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", "-o", LIB + ".tmp", SRC]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class OImage(C.Structure):
    _fields_ = [("band", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("npsf", C.c_int32), ("pixels", C.c_void_p), ("sky_map", C.c_void_p),
                ("sky", C.c_double), ("calib", C.c_double), ("wcs", C.c_double * 6),
                ("psf", C.c_void_p)]


class OProblem(C.Structure):
    _fields_ = [("n_img", C.c_int32), ("imgs", C.POINTER(OImage)),
                ("n_exp", C.c_int32), ("n_dev", C.c_int32),
                ("exp_mix", C.c_void_p), ("dev_mix", C.c_void_p),
                ("prior_star", C.c_double), ("prior_r", C.c_void_p),
                ("n_comp", C.c_int32), ("prior_c", C.c_void_p),
                ("n_src", C.c_int32), ("patch_off", C.c_void_p), ("patches", C.c_void_p),
                ("nbr_off", C.c_void_p), ("nbrs", C.c_void_p), ("patch_wcs", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """Holds a problem in the oracle's flat layout (keeps the arrays alive)."""

    def __init__(self, prob):
        self.prob = prob
        self._keep = []
        imgs = (OImage * len(prob.images))()
        for i, im in enumerate(prob.images):
            px = np.ascontiguousarray(im.pixels, dtype=np.float32)
            psf = np.ascontiguousarray(im.psf, dtype=np.float64)
            sm = None if im.sky_map is None else np.ascontiguousarray(im.sky_map, np.float32)
            self._keep += [px, psf, sm]
            imgs[i].band, imgs[i].height, imgs[i].width = im.band, px.shape[0], px.shape[1]
            imgs[i].npsf = psf.shape[0]
            imgs[i].pixels, imgs[i].sky_map = _ptr(px), _ptr(sm)
            imgs[i].sky, imgs[i].calib = im.sky, im.calib
            for k in range(6):
                imgs[i].wcs[k] = float(im.wcs[k])
            imgs[i].psf = _ptr(psf)
        self._imgs = imgs
        arrs = dict(
            exp_mix=np.ascontiguousarray(prob.exp_mix, np.float64),
            dev_mix=np.ascontiguousarray(prob.dev_mix, np.float64),
            prior_r=np.ascontiguousarray(prob.prior_r, np.float64),
            prior_c=np.ascontiguousarray(prob.prior_c, np.float64),
            patch_off=np.ascontiguousarray(prob.patch_offsets, np.int32),
            patches=np.ascontiguousarray(prob.patches, np.int32),
            nbr_off=np.ascontiguousarray(prob.nbr_offsets, np.int32),
            nbrs=np.ascontiguousarray(prob.nbrs, np.int32) if len(prob.nbrs) else np.zeros(1, np.int32),
        )
        self._arrs = arrs
        p = OProblem()
        p.n_img = len(prob.images)
        p.imgs = C.cast(imgs, C.POINTER(OImage))
        p.n_exp, p.n_dev = arrs["exp_mix"].shape[0], arrs["dev_mix"].shape[0]
        p.exp_mix, p.dev_mix = _ptr(arrs["exp_mix"]), _ptr(arrs["dev_mix"])
        p.prior_star = prob.prior_star
        p.prior_r = _ptr(arrs["prior_r"])
        p.n_comp = arrs["prior_c"].shape[1]
        p.prior_c = _ptr(arrs["prior_c"])
        p.n_src = prob.theta.shape[0]
        for k in ("patch_off", "patches", "nbr_off", "nbrs"):
            setattr(p, k, _ptr(arrs[k]))
        pw = getattr(prob, "patch_wcs", None)
        if pw is not None:
            arrs["patch_wcs"] = np.ascontiguousarray(pw, np.float64).reshape(-1, 6)
            assert arrs["patch_wcs"].shape[0] == arrs["patches"].shape[0]
            p.patch_wcs = _ptr(arrs["patch_wcs"])
        self.p = p
        self.L = lib()

    def _th(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        assert th.shape == (self.prob.n_src, NP_)
        return th

    def elbo(self, theta, maps=False):
        """Total ELBO over the union of patches and the local ELBO of each source."""
        th = self._th(theta)
        tot = C.c_double()
        loc = np.zeros(th.shape[0])
        npx = sum(im.pixels.size for im in self.prob.images)
        em = np.zeros(npx) if maps else None
        vm = np.zeros(npx) if maps else None
        rc = self.L.oracle_elbo(C.byref(self.p), _ptr(th), C.byref(tot), _ptr(loc), _ptr(em), _ptr(vm))
        if rc != 0:
            raise ValueError(f"oracle_elbo failed: {rc}")
        if maps:
            return tot.value, loc, em, vm
        return tot.value, loc

    def derivs(self, theta, which=None, hess=False):
        """(local ELBO, gradient [n][44], Hessian [n][44][44] or None) of each source."""
        th = self._th(theta)
        w = None if which is None else np.ascontiguousarray(which, np.int32)
        n = th.shape[0] if w is None else len(w)
        loc = np.zeros(n)
        g = np.zeros((n, NP_))
        h = np.zeros((n, NP_, NP_)) if hess else None
        rc = self.L.oracle_derivs(C.byref(self.p), _ptr(th), _ptr(w), C.c_int(n),
                                  C.c_int(1 if hess else 0), _ptr(loc), _ptr(g), _ptr(h))
        if rc != 0:
            raise ValueError(f"oracle_derivs failed: {rc}")
        return loc, g, h

    def kl(self, theta):
        th = self._th(theta)
        out = np.zeros(th.shape[0])
        rc = self.L.oracle_kl(C.byref(self.p), _ptr(th), _ptr(out))
        if rc != 0:
            raise ValueError(rc)
        return out

    def patch_values(self, theta, p):
        th = self._th(theta)
        w, h = int(self.prob.patches[p, 3]), int(self.prob.patches[p, 4])
        e = np.zeros(w * h)
        e2 = np.zeros(w * h)
        self.L.oracle_patch_values(C.byref(self.p), _ptr(th), C.c_int(p), _ptr(e), _ptr(e2))
        return e.reshape(h, w), e2.reshape(h, w)

    def profiles(self, theta_s, image, px, py):
        th = np.ascontiguousarray(theta_s, np.float64)
        px = np.ascontiguousarray(px, np.float64).ravel()
        py = np.ascontiguousarray(py, np.float64).ravel()
        gs = np.zeros(px.size)
        gg = np.zeros(px.size)
        self.L.oracle_profiles(C.byref(self.p), _ptr(th), C.c_int(image), C.c_int(px.size),
                               _ptr(px), _ptr(py), _ptr(gs), _ptr(gg))
        return gs, gg

    def colouring(self):
        col = np.zeros(self.prob.n_src, np.int32)
        nc = self.L.oracle_colouring(C.byref(self.p), _ptr(col))
        return col, nc

    def cyclades_batches(self, order, sample_size):
        """(batch_of, comp_of, n_batches) of one order under the Cyclades schedule."""
        od = np.ascontiguousarray(order, np.int32)
        b = np.zeros(len(od), np.int32)
        c = np.zeros(len(od), np.int32)
        nb = self.L.oracle_cyclades_batches(C.byref(self.p), _ptr(od), C.c_int(len(od)),
                                            C.c_int(sample_size), _ptr(c), _ptr(b))
        return b, c, nb

    def fit(self, theta, which=None, max_iter=50, grad_tol=1e-8, pred_tol_rel=1e-12,
            delta0=1.0, delta_max=1e3, eta=1e-4, f_noise_rel=1e-13, max_sweeps=20,
            sweep_tol=1e-8, order=None, sample_size=64):
        """Block-coordinate fit; with `order` ([max_sweeps][n_moving] permutations of the
        moving sources) the Cyclades schedule with samples of `sample_size`, else the
        colour schedule."""
        th = self._th(theta).copy()
        w = None if which is None else np.ascontiguousarray(which, np.int32)
        it = np.zeros(th.shape[0], np.int32)
        st = np.zeros(th.shape[0], np.int32)
        el = C.c_double()
        sw = C.c_int32()
        od = None
        if order is not None:
            od = np.ascontiguousarray(order, np.int32)
            n_moving = th.shape[0] if w is None else len(w)
            assert od.shape == (max_sweeps, n_moving)
        rc = self.L.oracle_fit(C.byref(self.p), _ptr(th), _ptr(w),
                               C.c_int(0 if w is None else len(w)), C.c_int(max_iter),
                               C.c_double(grad_tol), C.c_double(pred_tol_rel),
                               C.c_double(delta0), C.c_double(delta_max), C.c_double(eta),
                               C.c_double(f_noise_rel), C.c_int(max_sweeps),
                               C.c_double(sweep_tol), _ptr(it), _ptr(st), C.byref(el),
                               C.byref(sw), C.c_int(0 if order is None else 1),
                               C.c_int(sample_size), _ptr(od))
        if rc != 0:
            raise ValueError(f"oracle_fit failed: {rc}")
        return th, it, st, el.value, sw.value


def brightness(theta_s, band, i):
    L = lib()
    th = np.ascontiguousarray(theta_s, np.float64)
    a, b = C.c_double(), C.c_double()
    L.oracle_brightness(_ptr(th), C.c_int(band), C.c_int(i), C.byref(a), C.byref(b))
    return a.value, b.value


def to_free(theta_s):
    t = np.zeros(NT_)
    lib().oracle_to_free(_ptr(np.ascontiguousarray(theta_s, np.float64)), _ptr(t))
    return t


def from_free(t, jac=False):
    th = np.zeros(NP_)
    J = np.zeros((NP_, NT_)) if jac else None
    lib().oracle_from_free(_ptr(np.ascontiguousarray(t, np.float64)), _ptr(th), _ptr(J))
    return (th, J) if jac else th


def free_derivs(t, g44, h44):
    gt = np.zeros(NT_)
    ht = np.zeros((NT_, NT_))
    lib().oracle_free_derivs(_ptr(np.ascontiguousarray(t, np.float64)),
                             _ptr(np.ascontiguousarray(g44, np.float64)),
                             _ptr(np.ascontiguousarray(h44, np.float64)), _ptr(gt), _ptr(ht))
    return gt, ht


def tr_solve(c, B, delta):
    c = np.ascontiguousarray(c, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    p = np.zeros(c.size)
    pn = C.c_double()
    lib().oracle_tr_solve(C.c_int(c.size), _ptr(c), _ptr(B), C.c_double(delta), _ptr(p), C.byref(pn))
    return p, pn.value


def num_threads():
    return lib().oracle_num_threads()


def set_threads(n):
    lib().oracle_set_threads(C.c_int(n))
