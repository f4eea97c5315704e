"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on the
same seeded inputs.  Tolerances: FP64 path ELBO rel <= 1e-10, gradient rel-L2 <= 1e-8;
FP32-per-pixel path ELBO rel <= 1e-5, gradient rel-L2 <= 1e-4."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = {0: (1e-10, 1e-10, 1e-8), 1: (1e-5, 1e-5, 1e-4)}   # total, local, grad


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _check_problem(cel, prob, which=None):
    orc = Oracle(prob)
    o_tot, o_loc = orc.elbo(prob.theta)
    o_locd, o_g, _ = orc.derivs(prob.theta, which=which)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        te, tl, tg = TOL[prec]
        tot, loc = P.elbo(prob.theta, precision=prec)
        assert rel(tot, o_tot) <= te, (prec, tot, o_tot)
        assert np.max(np.abs(loc - o_loc) / np.abs(o_loc)) <= tl
        tot2, loc2, g = P.elbo_grad(prob.theta, precision=prec)
        assert rel(tot2, o_tot) <= te
        gs = g if which is None else g[which]
        ls = loc2 if which is None else loc2[which]
        assert np.max(np.abs(ls - o_locd) / np.abs(o_locd)) <= tl
        assert rel_l2(gs, o_g) <= tg, (prec, rel_l2(gs, o_g))
        # every source separately as well (no source hidden behind a larger one)
        for k in range(gs.shape[0]):
            assert rel_l2(gs[k], o_g[k]) <= 10 * tg, (prec, k, rel_l2(gs[k], o_g[k]))
    P.close()


def test_tiny_two_source(cel):
    _check_problem(cel, synth.config(0))


def test_crowded_region(cel):
    _check_problem(cel, synth.config(2))


def test_one_field_full_size_sampled(cel):
    """The benchmark's workload at full size (500 sources, 5 x 2048 x 1489): totals and
    local objectives of every source, gradients of a seeded sample of sources."""
    prob = synth.config(1)
    which = np.sort(np.random.default_rng(7).choice(prob.n_src, 24, replace=False)).astype(np.int32)
    _check_problem(cel, prob, which=which)


def test_edge_cases(cel):
    """Clipped patches at the image border, a one-pixel patch, a source with no patch
    (KL only), a sky map, a rotated WCS and ragged work-item tails."""
    th = np.stack([H.star_theta(1.0, 2.0), H.star_theta(20.0, 21.0, a_star=0.3),
                   H.star_theta(10.0, 10.0), H.star_theta(30.0, 5.0)])
    th[1, synth.I_AXIS] = 0.35
    patches = (np.array([0, 3, 8, 9, 9], np.int32),
               np.array([(0, 0, 0, 9, 11), (1, 0, 0, 17, 5), (4, 0, 0, 3, 1),
                         (0, 10, 12, 23, 20), (1, 10, 12, 22, 19), (2, 5, 5, 27, 27),
                         (3, 12, 14, 20, 18), (4, 13, 13, 19, 19),
                         (2, 10, 10, 1, 1)], np.int32))
    prob = H.problem(th, H=33, W=35, patches=patches, wcs=[0.98, -0.05, 0.05, 0.98, 0.7, -0.4])
    prob.images[2].sky_map = np.random.default_rng(3).uniform(120, 180, (33, 35)).astype(np.float32)
    _check_problem(cel, prob)


def test_autotuned_variants_agree(cel):
    """Every register budget of the item kernel gives the oracle's value and gradient, and
    every map-pass kernel code the oracle's gradient through the Hessian path, within the
    FP32 tolerances; the tuner returns one of them."""
    prob = synth.config(2)
    orc = Oracle(prob)
    o_tot, _ = orc.elbo(prob.theta)
    _, o_g, _ = orc.derivs(prob.theta)
    P = cel.Problem(prob)
    for code in (1, 2, 3, 4, 5):
        P.set_tuning(2, code)
        tot, loc, g = P.elbo_grad(prob.theta, precision=cel.FP32)
        assert rel(tot, o_tot) <= 1e-5 and rel_l2(g, o_g) <= 1e-4, code
    for code in (1, 2, 3, 4, 5, 6, 7):
        P.set_tuning(code, 0)
        _, g, _ = P.hess(prob.theta, precision=cel.FP32)
        assert rel_l2(g, o_g) <= 1e-4, code
    c, i = P.autotune(prob.theta)
    assert c in range(1, 8) and i in range(1, 6)
    with pytest.raises(cel.CelesteError):
        P.set_tuning(2, 6)
    with pytest.raises(cel.CelesteError):
        P.set_tuning(8, 0)
    P.close()


def test_device_entry_points_match_host(cel):
    import torch
    prob = synth.config(2)
    P = cel.Problem(prob)
    tot, loc, g = P.elbo_grad(prob.theta, precision=cel.FP32)
    dth = torch.tensor(prob.theta, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dl = torch.zeros(prob.n_src, dtype=torch.float64, device="cuda")
    dg = torch.zeros(prob.n_src, 44, dtype=torch.float64, device="cuda")
    P.elbo_grad_device(dth, dt, dl, dg, precision=cel.FP32)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    assert dt.item() == tot
    np.testing.assert_array_equal(dl.cpu().numpy(), loc)
    np.testing.assert_array_equal(dg.cpu().numpy(), g)
    # repeated calls are bit-identical (no atomics in any sum)
    P.elbo_grad_device(dth, dt, dl, dg, precision=cel.FP32)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dg.cpu().numpy(), g)
    P.close()


def test_page_locked_host_calls_match_pageable(cel):
    """The host-pointer call with page-locked host buffers (as the bench's end-to-end leg
    uses them): the same bits as with pageable buffers, the buffers re-read on every
    call, and a domain error still reported."""
    import ctypes as C
    import torch
    prob = synth.config(2)
    P = cel.Problem(prob)
    n = prob.n_src
    th = torch.tensor(prob.theta, dtype=torch.float64).pin_memory()
    tot = torch.zeros(1, dtype=torch.float64).pin_memory()
    loc = torch.zeros(n, dtype=torch.float64).pin_memory()
    g = torch.zeros(n, 44, dtype=torch.float64).pin_memory()

    def call():
        return P.L.celeste_elbo_grad(P.h, C.c_void_p(th.data_ptr()), cel.FP32, C.c_void_p(tot.data_ptr()),
                                     C.c_void_p(loc.data_ptr()), C.c_void_p(g.data_ptr()))

    for theta in (prob.theta, prob.theta * np.where(np.arange(44) == synth.I_R1, 1.01, 1.0)):
        th.copy_(torch.from_numpy(theta))
        for _ in range(2):
            assert call() == 0
            t0, l0, g0 = P.elbo_grad(theta, precision=cel.FP32)   # pageable buffers
            assert tot.item() == t0
            np.testing.assert_array_equal(loc.numpy(), l0)
            np.testing.assert_array_equal(g.numpy(), g0)
    bad = prob.theta.copy()
    bad[1, synth.I_R2] = -1.0
    th.copy_(torch.from_numpy(bad))
    assert call() == cel.ERR_ARG
    th.copy_(torch.from_numpy(prob.theta))
    assert call() == 0
    P.close()


def test_parameter_domain_boundaries(cel):
    """The device's domain check at the edges of each interval (it compares the doubles'
    bit patterns): e_dev in [0, 1] (-0 and 1 accepted), e_axis in (0, 1] (0 rejected, 1
    accepted), a in (0, 1) (1 rejected), variances > 0 (the smallest subnormal accepted,
    +0 rejected), Inf and NaN non-finite.  Checked through the device entry point, whose
    status the host reads."""
    import torch
    prob = synth.config(0)
    P = cel.Problem(prob)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    cases = [(synth.I_EDEV, -0.0, cel.OK), (synth.I_EDEV, 1.0, cel.OK), (synth.I_EDEV, np.nextafter(1.0, 2.0), cel.ERR_ARG),
             (synth.I_EDEV, -1e-300, cel.ERR_ARG), (synth.I_AXIS, 0.0, cel.ERR_ARG), (synth.I_AXIS, 1.0, cel.OK),
             (synth.I_AXIS, 5e-324, cel.OK), (synth.I_R2, 5e-324, cel.OK), (synth.I_R2, 0.0, cel.ERR_ARG),
             (synth.I_R2, -0.0, cel.ERR_ARG), (synth.I_R2, np.inf, cel.ERR_NONFINITE),
             (synth.I_R1, -np.inf, cel.ERR_NONFINITE), (synth.I_R1, np.nan, cel.ERR_NONFINITE)]
    for j, v, want in cases:
        th = prob.theta.copy()
        th[1, j] = v
        P.elbo_device(torch.tensor(th, dtype=torch.float64, device="cuda"), dt)
        torch.cuda.synchronize()
        assert P.device_status() == want, (j, v, P.device_status(), want)
    th = prob.theta.copy()
    th[1, synth.I_A] = 1.0
    th[1, synth.I_A + 1] = 0.0
    P.elbo_device(torch.tensor(th, dtype=torch.float64, device="cuda"), dt)
    torch.cuda.synchronize()
    assert P.device_status() == cel.ERR_ARG
    P.close()


def test_invalid_parameters_are_errors_not_faults(cel):
    import torch
    prob = synth.config(0)
    P = cel.Problem(prob)
    bad = prob.theta.copy()
    bad[1, synth.I_R2] = -1.0
    with pytest.raises(cel.CelesteError) as e:
        P.elbo(bad)
    assert e.value.status == cel.ERR_ARG
    bad2 = prob.theta.copy()
    bad2[0, 3] = np.nan
    with pytest.raises(cel.CelesteError) as e:
        P.elbo_grad(bad2)
    assert e.value.status == cel.ERR_NONFINITE
    dth = torch.tensor(bad, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.elbo_device(dth, dt)
    assert P.device_status() == cel.ERR_ARG
    # the problem stays usable
    tot, _ = P.elbo(prob.theta)
    assert np.isfinite(tot)
    P.close()


def test_bad_problem_inputs_rejected(cel):
    prob = synth.config(0)
    prob.images[0].psf = prob.images[0].psf.copy()
    prob.images[0].psf[0, 3] = -1.0
    with pytest.raises(cel.CelesteError) as e:
        cel.Problem(prob)
    assert e.value.status == cel.ERR_NOT_PD
    prob = synth.config(0)
    prob.patches = prob.patches.copy()
    prob.patches[0, 3] = 500
    with pytest.raises(cel.CelesteError) as e:
        cel.Problem(prob)
    assert e.value.status == cel.ERR_ARG


HTOL = {0: 1e-8, 1: 1e-4}


def _check_hessian(cel, prob, which=None):
    orc = Oracle(prob)
    o_loc, o_g, o_h = orc.derivs(prob.theta, which=which, hess=True)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        loc, g, h = P.hess(prob.theta, precision=prec)
        if which is not None:
            loc, g, h = loc[which], g[which], h[which]
        te, tl, tg = TOL[prec]
        assert np.max(np.abs(loc - o_loc) / np.abs(o_loc)) <= tl
        assert rel_l2(g, o_g) <= tg
        for k in range(h.shape[0]):
            assert np.abs(h[k] - h[k].T).max() <= 1e-12 * np.abs(h[k]).max()
            assert rel_l2(h[k], o_h[k]) <= HTOL[prec], (prec, k, rel_l2(h[k], o_h[k]))
    P.close()


def test_hessian_tiny(cel):
    _check_hessian(cel, synth.config(0))


def test_hessian_crowded(cel):
    _check_hessian(cel, synth.config(2), which=np.arange(0, 64, 4).astype(np.int32))


def test_hessian_one_field_full_size_sampled(cel):
    """The benchmark's workload at full size (500 sources, 5 x 2048 x 1489): local
    objectives, gradients and 44 x 44 Hessians of the seeded sample of 24 sources the
    gradient test uses, both precisions."""
    prob = synth.config(1)
    which = np.sort(np.random.default_rng(7).choice(prob.n_src, 24, replace=False)).astype(np.int32)
    _check_hessian(cel, prob, which=which)


def test_hessian_edge_cases(cel):
    th = np.stack([H.star_theta(1.0, 2.0), H.star_theta(20.0, 21.0, a_star=0.3)])
    th[1, synth.I_AXIS] = 0.35
    patches = (np.array([0, 3, 6], np.int32),
               np.array([(0, 0, 0, 9, 11), (1, 0, 0, 17, 5), (4, 0, 0, 3, 1),
                         (0, 10, 12, 23, 20), (2, 5, 5, 27, 27), (4, 13, 13, 19, 19)], np.int32))
    prob = H.problem(th, H=33, W=35, patches=patches, wcs=[0.98, -0.05, 0.05, 0.98, 0.7, -0.4])
    _check_hessian(cel, prob)
