"""Thin Python binding of libceleste (the C ABI in include/celeste.h).

Argument marshalling only: every step of the ELBO / gradient / Hessian / fit path
runs in the library's CUDA kernels.  Host-pointer calls take numpy arrays; the
``*_device`` calls take CUDA torch tensors and enqueue on torch's current stream.
There is no CPU fallback: when the shared library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NPARAM = 44
NFREE = 41
FP64 = 0
FP32 = 1          # FP32 per-pixel arithmetic, FP64 accumulation
SCHED_COLOUR = 0    # fit schedule: one batch per colour of a greedy colouring
SCHED_CYCLADES = 1  # fit schedule: connected components of random samples

OK, ERR_ARG, ERR_NOT_PD, ERR_NONFINITE, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6, -7


class CelesteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"celeste status {status}: {msg}")
        self.status = status


class celeste_image(C.Structure):
    _fields_ = [("band", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("pixels", C.c_void_p), ("sky", C.c_double), ("sky_map", C.c_void_p),
                ("nmgy_per_count", C.c_double), ("wcs", C.c_double * 6),
                ("n_psf", C.c_int32), ("psf", C.c_void_p)]


class celeste_model(C.Structure):
    _fields_ = [("n_exp", C.c_int32), ("n_dev", C.c_int32), ("exp_mix", C.c_void_p),
                ("dev_mix", C.c_void_p), ("prior_star", C.c_double), ("prior_r", C.c_void_p),
                ("n_color_comp", C.c_int32), ("prior_c", C.c_void_p)]


class celeste_patch(C.Structure):
    _fields_ = [("image", C.c_int32), ("x0", C.c_int32), ("y0", C.c_int32), ("w", C.c_int32),
                ("h", C.c_int32)]


class celeste_fit_options(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("grad_tol", C.c_double), ("pred_tol_rel", C.c_double),
                ("delta0", C.c_double), ("delta_max", C.c_double), ("eta", C.c_double),
                ("f_noise_rel", C.c_double), ("precision", C.c_int32), ("max_sweeps", C.c_int32),
                ("sweep_tol", C.c_double), ("refine_fp64", C.c_int32), ("schedule", C.c_int32),
                ("sample_size", C.c_int32), ("seed", C.c_uint64), ("order", C.c_void_p)]


_lib = None

EXPORTS = ["celeste_problem_create", "celeste_problem_create_ex", "celeste_problem_destroy",
           "celeste_source_pixels",
           "celeste_problem_stats",
           "celeste_elbo", "celeste_elbo_grad", "celeste_hess", "celeste_fit_options_default",
           "celeste_fit_sources", "celeste_elbo_device", "celeste_elbo_grad_device",
           "celeste_hess_device", "celeste_device_status", "celeste_last_error",
           "celeste_profile_enable", "celeste_profile_read",
           "celeste_patch_elbo_grad_noalloc", "celeste_grad_device", "celeste_autotune",
           "celeste_set_tuning", "celeste_cyclades_batches", "celeste_catalog",
           "celeste_catalog_device", "celeste_catalog_score", "celeste_render",
           "celeste_render_device", "celeste_make_tasks", "celeste_fit_tasks",
           "celeste_selftest_bounded_wait"]

# catalog row layout (CELESTE_CAT_*): position, type, per-type brightness / colours with
# their posterior standard deviations, the type-marginal r flux, galaxy shape
_COL = ("ug", "gr", "ri", "iz")
_TYPE_FIELDS = (["rmag", "rmag_sd", "rflux", "rflux_sd"] + [f"color_{c}" for c in _COL]
                + [f"color_{c}_sd" for c in _COL] + [f"mag_{b}" for b in "ugriz"]
                + [f"mag_{b}_sd" for b in "ugriz"])
CAT_FIELDS = (["u0", "u1", "p_star", "is_star"] + [f"star_{f}" for f in _TYPE_FIELDS]
              + [f"gal_{f}" for f in _TYPE_FIELDS]
              + ["rflux_mix", "rflux_mix_sd", "e_dev", "e_axis", "angle_deg", "scale"])
CAT_NFIELD = len(CAT_FIELDS)
SCORE_FIELDS = ["position", "missed_gal", "missed_star", "brightness"] + \
    [f"color_{c}" for c in _COL] + ["profile", "axis", "scale", "angle_deg", "n_gal", "n_star"]


def lib_path():
    """The library the binding loads: the checked build (device-side bounds checks) when
    the environment sets CELESTE_CHECK_BOUNDS=1, else the normal build."""
    return _build.LIB_CHECKED if os.environ.get("CELESTE_CHECK_BOUNDS") == "1" else _build.LIB


def load(build_if_missing=False):
    """Load libceleste.  Raises when the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build(checked=path == _build.LIB_CHECKED)
        else:
            raise RuntimeError(f"libceleste is not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    L.celeste_problem_create.argtypes = [C.POINTER(celeste_image), i32, C.POINTER(celeste_model), i32,
                                         vp, C.POINTER(celeste_patch), vp, vp, C.POINTER(vp)]
    L.celeste_problem_create.restype = i32
    L.celeste_problem_create_ex.argtypes = [C.POINTER(celeste_image), i32, C.POINTER(celeste_model), i32,
                                            vp, C.POINTER(celeste_patch), vp, vp, vp, C.POINTER(vp)]
    L.celeste_problem_create_ex.restype = i32
    L.celeste_problem_destroy.argtypes = [vp]
    L.celeste_problem_destroy.restype = None
    L.celeste_source_pixels.argtypes = [vp]
    L.celeste_source_pixels.restype = i64
    L.celeste_problem_stats.argtypes = [vp, vp, C.c_int32]
    L.celeste_problem_stats.restype = C.c_int32
    L.celeste_elbo.argtypes = [vp, vp, i32, vp, vp]
    L.celeste_elbo_grad.argtypes = [vp, vp, i32, vp, vp, vp]
    L.celeste_hess.argtypes = [vp, vp, i32, vp, vp, vp]
    for f in ("celeste_elbo", "celeste_elbo_grad", "celeste_hess"):
        getattr(L, f).restype = i32
    L.celeste_fit_options_default.argtypes = [C.POINTER(celeste_fit_options)]
    L.celeste_fit_options_default.restype = None
    L.celeste_fit_sources.argtypes = [vp, vp, vp, i32, C.POINTER(celeste_fit_options), vp, vp, vp]
    L.celeste_fit_sources.restype = i32
    L.celeste_elbo_device.argtypes = [vp, vp, i32, vp, vp, vp]
    L.celeste_elbo_grad_device.argtypes = [vp, vp, i32, vp, vp, vp, vp]
    L.celeste_hess_device.argtypes = [vp, vp, i32, vp, vp, vp, vp]
    for f in ("celeste_elbo_device", "celeste_elbo_grad_device", "celeste_hess_device"):
        getattr(L, f).restype = i32
    L.celeste_grad_device.argtypes = [vp, vp, i32, vp, vp, vp]
    L.celeste_grad_device.restype = i32
    L.celeste_autotune.argtypes = [vp, vp, i32, vp, vp]
    L.celeste_autotune.restype = i32
    L.celeste_set_tuning.argtypes = [vp, i32, i32]
    L.celeste_set_tuning.restype = i32
    L.celeste_cyclades_batches.argtypes = [vp, vp, i32, vp, i32, i32, vp, vp, vp]
    L.celeste_cyclades_batches.restype = i32
    L.celeste_catalog.argtypes = [vp, vp, vp]
    L.celeste_catalog_device.argtypes = [vp, vp, vp, vp]
    L.celeste_catalog_score.argtypes = [vp, vp, vp, i32, vp]
    L.celeste_selftest_bounded_wait.argtypes = []
    L.celeste_selftest_bounded_wait.restype = i32
    L.celeste_make_tasks.argtypes = [vp, vp, i32, C.c_double, vp, vp, vp]
    L.celeste_make_tasks.restype = i32
    L.celeste_fit_tasks.argtypes = [vp, vp, vp, C.POINTER(celeste_fit_options), vp, vp, vp]
    L.celeste_fit_tasks.restype = i32
    L.celeste_render.argtypes = [vp, vp, vp, vp]
    L.celeste_render_device.argtypes = [vp, vp, vp, vp, vp]
    for f in ("celeste_catalog", "celeste_catalog_device", "celeste_catalog_score", "celeste_render",
              "celeste_render_device"):
        getattr(L, f).restype = i32
    L.celeste_device_status.argtypes = [vp]
    L.celeste_device_status.restype = i32
    L.celeste_profile_enable.argtypes = [vp, i32]
    L.celeste_profile_enable.restype = i32
    L.celeste_profile_read.argtypes = [vp, i32, vp, vp, vp]
    L.celeste_profile_read.restype = i32
    L.celeste_patch_elbo_grad_noalloc.argtypes = [C.POINTER(celeste_image), C.POINTER(celeste_model),
                                                  C.POINTER(celeste_patch), vp, vp, vp, i32, vp,
                                                  vp, vp, vp]
    L.celeste_patch_elbo_grad_noalloc.restype = i32
    L.celeste_last_error.argtypes = []
    L.celeste_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(st):
    if st != OK:
        raise CelesteError(st, _lib.celeste_last_error().decode())


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def cyclades_batches(nbr_offsets, nbrs, order, sample_size):
    """Batch of each position of `order`, and the order position of the first member of
    its component, under the Cyclades schedule over the neighbour graph (CSR); returns
    (batch_of, comp_of, n_batches).  Host logic: no CUDA device needed."""
    L = load()
    no = np.ascontiguousarray(nbr_offsets, np.int32)
    nb_ = np.ascontiguousarray(nbrs, np.int32)
    order = np.ascontiguousarray(order, np.int32)
    b = np.zeros(len(order), np.int32)
    c = np.zeros(len(order), np.int32)
    nb = C.c_int32()
    _check(L.celeste_cyclades_batches(_p(no), _p(nb_), len(no) - 1, _p(order), len(order),
                                      int(sample_size), _p(b), _p(c), C.byref(nb)))
    return b, c, nb.value


def selftest_bounded_wait():
    """Status of the bounded-wait self-test (ERR_TIMEOUT expected; see celeste.h)."""
    return int(load().celeste_selftest_bounded_wait())


def make_tasks(pos, work, max_work, shift=None):
    """Region tasks of one stage: (task of every source, number of tasks).  Host logic:
    no CUDA device needed."""
    L = load()
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 2)
    work = np.ascontiguousarray(work, np.float64)
    out = np.zeros(pos.shape[0], np.int32)
    sh = None if shift is None else np.ascontiguousarray(shift, np.float64)
    nt = C.c_int32()
    _check(L.celeste_make_tasks(_p(pos), _p(work), pos.shape[0], float(max_work), _p(sh), _p(out),
                                C.byref(nt)))
    return out, nt.value


def fit_options(**kw):
    o = celeste_fit_options()
    load().celeste_fit_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Problem:
    """A Celeste problem resident on the current CUDA device (owns its device copy)."""

    def __init__(self, prob):
        L = load()
        self.n_src = int(prob.theta.shape[0])
        self.shapes = [tuple(im.pixels.shape) for im in prob.images]
        keep = []
        imgs = (celeste_image * len(prob.images))()
        for i, im in enumerate(prob.images):
            px = np.ascontiguousarray(im.pixels, np.float32)
            psf = np.ascontiguousarray(im.psf, np.float64)
            sm = None if im.sky_map is None else np.ascontiguousarray(im.sky_map, np.float32)
            keep += [px, psf, sm]
            imgs[i].band, imgs[i].height, imgs[i].width = im.band, px.shape[0], px.shape[1]
            imgs[i].pixels, imgs[i].sky, imgs[i].sky_map = _p(px), float(im.sky), _p(sm)
            imgs[i].nmgy_per_count = float(im.calib)
            for k in range(6):
                imgs[i].wcs[k] = float(im.wcs[k])
            imgs[i].n_psf, imgs[i].psf = psf.shape[0], _p(psf)
        exp_mix = np.ascontiguousarray(prob.exp_mix, np.float64)
        dev_mix = np.ascontiguousarray(prob.dev_mix, np.float64)
        prior_r = np.ascontiguousarray(prob.prior_r, np.float64)
        prior_c = np.ascontiguousarray(prob.prior_c, np.float64)
        keep += [exp_mix, dev_mix, prior_r, prior_c]
        m = celeste_model(exp_mix.shape[0], dev_mix.shape[0], _p(exp_mix), _p(dev_mix),
                          float(prob.prior_star), _p(prior_r), prior_c.shape[1], _p(prior_c))
        po = np.ascontiguousarray(prob.patch_offsets, np.int32)
        pa = np.ascontiguousarray(prob.patches, np.int32).reshape(-1, 5)
        patches = (celeste_patch * max(1, pa.shape[0]))()
        for i in range(pa.shape[0]):
            patches[i] = celeste_patch(*(int(v) for v in pa[i]))
        no = np.ascontiguousarray(prob.nbr_offsets, np.int32)
        nb = np.ascontiguousarray(prob.nbrs, np.int32)
        keep += [po, no, nb]
        h = C.c_void_p()
        pw = getattr(prob, "patch_wcs", None)   # per-patch linearised maps (optional)
        if pw is not None:
            pw = np.ascontiguousarray(pw, np.float64).reshape(-1, 6)
            if pw.shape[0] != pa.shape[0]:
                raise ValueError("patch_wcs must hold one map per patch")
            keep.append(pw)
        st = L.celeste_problem_create_ex(imgs, len(prob.images), C.byref(m), self.n_src, _p(po),
                                         patches, _p(pw), _p(no), _p(nb) if nb.size else None,
                                         C.byref(h))
        _check(st)
        self.h = h
        self.L = L
        self.generation = 0    # bumped by every call that rebuilds the E / Var maps

    def close(self):
        if getattr(self, "h", None):
            self.L.celeste_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def source_pixels(self):
        return int(self.L.celeste_source_pixels(self.h))

    STAT_KEYS = ("sources", "patches", "items", "fp32_items", "single_source_pixels", "tiles",
                 "source_pixels", "other_evals")

    def stats(self):
        """Work decomposition: {sources, patches, items, fp32_items, single_source_pixels,
        tiles, source_pixels, other_evals}."""
        out = np.zeros(len(self.STAT_KEYS), np.int64)
        n = self.L.celeste_problem_stats(self.h, _p(out), len(out))
        if n < 0:
            _check(n)
        return {k: int(v) for k, v in zip(self.STAT_KEYS, out[:n])}

    def _theta(self, theta):
        th = np.ascontiguousarray(theta, np.float64)
        if th.shape != (self.n_src, NPARAM):
            raise ValueError(f"theta must be [{self.n_src}][{NPARAM}]")
        return th

    # ---- host-pointer calls
    def elbo(self, theta, precision=FP64):
        self.generation += 1   # the problem's maps now belong to this call
        th = self._theta(theta)
        tot = C.c_double()
        loc = np.zeros(self.n_src)
        _check(self.L.celeste_elbo(self.h, _p(th), precision, C.byref(tot), _p(loc)))
        return tot.value, loc

    def elbo_grad(self, theta, precision=FP64):
        self.generation += 1   # the problem's maps now belong to this call
        th = self._theta(theta)
        tot = C.c_double()
        loc = np.zeros(self.n_src)
        g = np.zeros((self.n_src, NPARAM))
        _check(self.L.celeste_elbo_grad(self.h, _p(th), precision, C.byref(tot), _p(loc), _p(g)))
        return tot.value, loc, g

    def hess(self, theta, precision=FP64):
        self.generation += 1   # the problem's maps now belong to this call
        th = self._theta(theta)
        loc = np.zeros(self.n_src)
        g = np.zeros((self.n_src, NPARAM))
        h = np.zeros((self.n_src, NPARAM, NPARAM))
        _check(self.L.celeste_hess(self.h, _p(th), precision, _p(loc), _p(g), _p(h)))
        return loc, g, h

    def fit(self, theta, which=None, **opts):
        self.generation += 1   # the problem's maps now belong to this call
        th = self._theta(theta).copy()
        w = None if which is None else np.ascontiguousarray(which, np.int32)
        it = np.zeros(self.n_src, np.int32)
        st = np.zeros(self.n_src, np.int32)
        el = C.c_double()
        order = opts.pop("order", None)
        if isinstance(opts.get("schedule"), str):
            opts["schedule"] = {"colour": SCHED_COLOUR, "cyclades": SCHED_CYCLADES}[opts["schedule"]]
        o = fit_options(**opts)
        if order is not None:
            order = np.ascontiguousarray(order, np.int32)
            o.order = order.ctypes.data
        _check(self.L.celeste_fit_sources(self.h, _p(th), _p(w), 0 if w is None else len(w),
                                          C.byref(o), _p(it), _p(st), C.byref(el)))
        return th, it, st, el.value


    def fit_tasks(self, theta, task_of, **opts):
        """One stage of region tasks (celeste_fit_tasks): (theta, iters, status, elbo)."""
        self.generation += 1
        th = self._theta(theta).copy()
        t = np.ascontiguousarray(task_of, np.int32)
        it = np.zeros(self.n_src, np.int32)
        st = np.zeros(self.n_src, np.int32)
        el = C.c_double()
        o = fit_options(**opts)
        _check(self.L.celeste_fit_tasks(self.h, _p(th), _p(t), C.byref(o), _p(it), _p(st), C.byref(el)))
        return th, it, st, el.value

    def render(self, theta):
        """The model's expected image E[F] and variance Var[F] at theta, one [H][W] array
        per image (FP64)."""
        th = self._theta(theta)
        npx = sum(h * w for h, w in self.shapes)
        e = np.zeros(npx, np.float64)
        v = np.zeros(npx, np.float64)
        _check(self.L.celeste_render(self.h, _p(th), _p(e), _p(v)))
        out_e, out_v, off = [], [], 0
        for h, w in self.shapes:
            out_e.append(e[off:off + h * w].reshape(h, w))
            out_v.append(v[off:off + h * w].reshape(h, w))
            off += h * w
        return out_e, out_v

    def catalog(self, theta):
        """Catalog rows [n_src][CAT_NFIELD] (columns named by CAT_FIELDS)."""
        th = self._theta(theta)
        out = np.zeros((self.n_src, CAT_NFIELD), np.float64)
        _check(self.L.celeste_catalog(self.h, _p(th), _p(out)))
        return out

    def catalog_score(self, cat_est, cat_true):
        """Table II style error summary of cat_est against cat_true: dict by SCORE_FIELDS."""
        e = np.ascontiguousarray(cat_est, np.float64)
        t = np.ascontiguousarray(cat_true, np.float64)
        assert e.shape == t.shape and e.shape[1:] == (CAT_NFIELD,)
        out = np.zeros(len(SCORE_FIELDS), np.float64)
        _check(self.L.celeste_catalog_score(self.h, _p(e), _p(t), e.shape[0], _p(out)))
        return dict(zip(SCORE_FIELDS, out.tolist()))

    def catalog_device(self, d_theta, d_cat):
        _check(self.L.celeste_catalog_device(self.h, self._dp(d_theta), self._dp(d_cat),
                                             self._stream()))

    # ---- device-pointer calls (torch tensors on the problem's device)
    @staticmethod
    def _stream():
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    @staticmethod
    def _dp(t):
        if t is None:
            return None
        assert t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous()
        return C.c_void_p(t.data_ptr())

    def elbo_device(self, d_theta, d_total, d_local=None, precision=FP32):
        self.generation += 1   # the problem's maps now belong to this call
        _check(self.L.celeste_elbo_device(self.h, self._dp(d_theta), precision, self._dp(d_total),
                                          self._dp(d_local), self._stream()))

    def elbo_grad_device(self, d_theta, d_total, d_local, d_grad, precision=FP32):
        self.generation += 1   # the problem's maps now belong to this call
        _check(self.L.celeste_elbo_grad_device(self.h, self._dp(d_theta), precision,
                                               self._dp(d_total), self._dp(d_local),
                                               self._dp(d_grad), self._stream()))

    def grad_device(self, d_theta, d_grad, d_local=None, precision=FP32):
        """Adjoint only; needs the preceding elbo_device call on the same theta."""
        _check(self.L.celeste_grad_device(self.h, self._dp(d_theta), precision, self._dp(d_local),
                                          self._dp(d_grad), self._stream()))

    def hess_device(self, d_theta, d_local, d_grad, d_hess, precision=FP32):
        self.generation += 1   # the problem's maps now belong to this call
        _check(self.L.celeste_hess_device(self.h, self._dp(d_theta), precision, self._dp(d_local),
                                          self._dp(d_grad), self._dp(d_hess), self._stream()))

    def autotune(self, theta, reps=5):
        """Pick the fastest FP32 kernel variants; returns (contrib code, items code)."""
        self.generation += 1
        out = [C.c_int32() for _ in range(2)]
        _check(self.L.celeste_autotune(self.h, _p(self._theta(theta)), reps,
                                       *(C.byref(o) for o in out)))
        return tuple(o.value for o in out)

    def set_tuning(self, contrib_code, items_code=0):
        _check(self.L.celeste_set_tuning(self.h, contrib_code, items_code))

    def profile(self, on=True, serial=False):
        """Per-stage CUDA-event timing; serial=True runs every stage on the calling
        stream, one after another."""
        _check(self.L.celeste_profile_enable(self.h, (2 if serial else 1) if on else 0))

    def profile_read(self):
        """{stage: (total ms, launches)} since the last read."""
        mx = 32
        names = C.create_string_buffer(32 * mx)
        ms = np.zeros(mx)
        n_l = np.zeros(mx, np.int32)
        n = self.L.celeste_profile_read(self.h, mx, names, _p(ms), _p(n_l))
        if n < 0:
            _check(n)
        raw = names.raw
        return {raw[32 * k:32 * k + 32].split(b"\0")[0].decode(): (float(ms[k]), int(n_l[k]))
                for k in range(n)}

    def device_status(self):
        return int(self.L.celeste_device_status(self.h))


def patch_elbo_grad_noalloc(image, exp_mix, dev_mix, prior_star, prior_r, prior_c, patch,
                            d_pixels, d_theta, d_total, d_local, d_grad, d_sky_map=None,
                            precision=FP64):
    """Allocation-free ELBO + gradient of one source confined to one patch.

    For callers that cannot call cudaMalloc (device memory owned by another
    allocator, or no allocation allowed on the calling path): every intermediate
    buffer lives in a fixed device array inside the library.  ``image`` is a
    ``synth.Image`` (its pixels are not read); ``patch`` is (x0, y0, w, h) in that
    image's pixel frame; the ``d_*`` arguments are CUDA torch tensors: the patch's
    pixels [h][w] float32, theta [44], and float64 outputs total [1], local [1],
    grad [44].  Work is enqueued on torch's current stream."""
    L = load()
    psf = np.ascontiguousarray(image.psf, np.float64)
    im = celeste_image()
    im.band, im.height, im.width = image.band, image.height, image.width
    im.pixels, im.sky, im.sky_map = None, float(image.sky), None
    im.nmgy_per_count = float(image.calib)
    for k in range(6):
        im.wcs[k] = float(image.wcs[k])
    im.n_psf, im.psf = psf.shape[0], _p(psf)
    em = np.ascontiguousarray(exp_mix, np.float64)
    dm = np.ascontiguousarray(dev_mix, np.float64)
    pr = np.ascontiguousarray(prior_r, np.float64)
    pc = np.ascontiguousarray(prior_c, np.float64)
    m = celeste_model(em.shape[0], dm.shape[0], _p(em), _p(dm), float(prior_star), _p(pr),
                      pc.shape[1], _p(pc))
    p = celeste_patch(0, *(int(v) for v in patch))
    import torch

    def ptr(t):
        return None if t is None else C.c_void_p(t.data_ptr())

    st = L.celeste_patch_elbo_grad_noalloc(C.byref(im), C.byref(m), C.byref(p), ptr(d_pixels),
                                           ptr(d_sky_map), ptr(d_theta), precision, ptr(d_total),
                                           ptr(d_local), ptr(d_grad),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(st)
