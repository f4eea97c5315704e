"""Block-coordinate trust-region Newton fits (Section IV-D) on the GPU against the
oracle's fit from the same starts: positions within 1e-3 px and r-band expected
fluxes within 1e-4 relative for sources both sides report converged, in both
precisions."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def rflux(th):
    """r-band expected flux E[l | i] of the more probable type i (nanomaggies): the
    catalog brightness.  The other type's brightness carries weight a_i ~ 0.005 at the
    optimum and is barely constrained by the data."""
    i = 0 if th[synth.I_A] >= th[synth.I_A + 1] else 1
    return np.exp(th[synth.I_R1 + i] + 0.5 * th[synth.I_R2 + i])


def _compare(cel, prob, which=None, max_sweeps=20, sweep_tol=1e-12):
    """Both sides sweep until the total ELBO stops moving (relative 1e-12): a looser
    sweep tolerance leaves overlapping sources short of the joint optimum by amounts
    that depend on the path."""
    orc = Oracle(prob)
    o_th, o_it, o_st, o_el, _ = orc.fit(prob.theta, which=which, max_sweeps=max_sweeps,
                                        sweep_tol=sweep_tol)
    P = cel.Problem(prob)
    moving = np.arange(prob.n_src) if which is None else np.asarray(which)
    for prec in (cel.FP64, cel.FP32):
        th, it, st, el = P.fit(prob.theta, which=which, precision=prec, max_sweeps=max_sweeps,
                               sweep_tol=sweep_tol)
        assert np.all(it[moving] <= 50 * max_sweeps * (2 if prec == cel.FP32 else 1))
        both = [s for s in moving if st[s] == 0 and o_st[s] == 0]
        assert len(both) >= 0.75 * len(moving), (prec, st[moving], o_st[moving])
        for s in both:
            assert np.abs(th[s, 0:2] - o_th[s, 0:2]).max() <= 1e-3, (prec, s, th[s, :2], o_th[s, :2])
            assert abs(rflux(th[s]) / rflux(o_th[s]) - 1) <= 1e-4, (prec, s, th[s], o_th[s])
        assert abs(el - o_el) <= (1e-8 if prec == cel.FP64 else 1e-5) * abs(o_el), (prec, el, o_el)
        # sources outside `which` never move
        still = np.setdiff1d(np.arange(prob.n_src), moving)
        np.testing.assert_array_equal(th[still], prob.theta[still])
    P.close()


def test_fit_tiny_two_sources(cel):
    _compare(cel, synth.config(0))


def independent_set(prob, k):
    """k sources no two of which overlap: with the others fixed, one block-coordinate
    sweep already reaches the optimum, so a fit from identical starts has one answer."""
    chosen = []
    for s in range(0, prob.n_src, 3):
        nb = set(prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]].tolist())
        if not nb & set(chosen):
            chosen.append(s)
        if len(chosen) == k:
            break
    return np.array(chosen, np.int32)


def test_fit_crowded_subset(cel):
    prob = synth.config(2)
    _compare(cel, prob, which=independent_set(prob, 8), max_sweeps=2)


def test_fit_rejects_parameters_outside_the_box(cel):
    prob = synth.config(0)
    P = cel.Problem(prob)
    bad = prob.theta.copy()
    bad[0, synth.I_A] = 0.999
    bad[0, synth.I_A + 1] = 0.001
    with pytest.raises(cel.CelesteError) as e:
        P.fit(bad)
    assert e.value.status == cel.ERR_ARG
    P.close()
