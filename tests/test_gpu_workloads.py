"""GPU parity on the large workloads, at full size, through the C ABI.

* Multi-epoch region (8 overlapping 2048 x 1489 fields, 5 bands each, per-image PSF,
  sky, calibration and affine WCS; 20,000 sources).  The oracle cannot evaluate every
  source in seconds, so a seeded sample of sources is checked one by one: the local
  objective of a source depends only on the pixels of its patches, where E and Var are
  sums over the sources whose patches cover them, i.e. the source and its neighbours.
  The oracle therefore runs on the sub-problem made of the sample and their
  neighbours, whose local objectives and gradients for the sampled sources are those of
  the full problem exactly.
* Sweep field (one of 64 disjoint fields: 3,125 sources, 10 % bright with patches up
  to 101 px).  The oracle evaluates the whole field; totals, every local objective and
  the gradients of a 1,000-source sample are compared.

* The whole sweep (the 64 fields as one 200,000-source problem): each field's sources
  against the same field evaluated alone.

Tolerances as in test_gpu_parity: FP64 path ELBO rel <= 1e-10, gradient rel-L2 <= 1e-8;
FP32 path ELBO rel <= 1e-5, gradient rel-L2 <= 1e-4.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests.helpers import neighbour_closure as closure

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


def test_multi_epoch_region_sampled(cel):
    prob = synth.config(3)
    assert prob.n_src == 20000 and len(prob.images) == 40
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(prob.n_src, 32, replace=False))
    keep = closure(prob, sample)
    sub = synth.subset(prob, keep)
    pos = np.searchsorted(keep, sample).astype(np.int32)
    o_l, o_g, _ = Oracle(sub).derivs(sub.theta, which=pos)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        _, tl, tg = TOL[prec]
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        assert np.isfinite(tot)
        assert np.max(np.abs(loc[sample] - o_l) / np.abs(o_l)) <= tl, prec
        assert rel_l2(g[sample], o_g) <= tg, (prec, rel_l2(g[sample], o_g))
        for k in range(len(sample)):
            assert rel_l2(g[sample[k]], o_g[k]) <= 10 * tg, (prec, k)
    P.close()


def test_sweep_field_with_bright_sources(cel):
    prob = synth.config(4)
    bright = np.flatnonzero(prob.patches[:, 3] >= 75)
    assert bright.size > 0    # the large patches are part of the case
    orc = Oracle(prob)
    o_tot, o_loc = orc.elbo(prob.theta)
    rng = np.random.default_rng(12)
    which = np.sort(rng.choice(prob.n_src, 1000, replace=False)).astype(np.int32)
    _, o_g, _ = orc.derivs(prob.theta, which=which)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        te, tl, tg = TOL[prec]
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        assert rel(tot, o_tot) <= te, (prec, tot, o_tot)
        assert np.max(np.abs(loc - o_loc) / np.abs(o_loc)) <= tl, prec
        assert rel_l2(g[which], o_g) <= tg, (prec, rel_l2(g[which], o_g))
    P.close()


def test_whole_sweep_matches_its_fields(cel):
    """The 200,000-source sweep as one problem (64 disjoint fields, 320 images): every
    source's local objective and gradient equal those of its field evaluated alone (the
    fields share no pixels; field 0 is the sweep field checked against the oracle above
    on 1,000 sampled sources), and the total is the sum of the fields' totals."""
    sweep = synth.config(6)
    assert sweep.n_src == 200000 and len(sweep.images) == 320
    P = cel.Problem(sweep)
    res = {prec: P.elbo_grad(sweep.theta, precision=prec) for prec in (cel.FP64, cel.FP32)}
    P.close()
    for f in (0, 37, 63):
        fld = synth.one_field(2030 + 7919 * f, n_src=3125, bright_frac=0.1)
        # the sweep shares field 0's priors (each field alone draws its own)
        fld.prior_star, fld.prior_r, fld.prior_c = sweep.prior_star, sweep.prior_r, sweep.prior_c
        rows = slice(3125 * f, 3125 * (f + 1))
        Pf = cel.Problem(fld)
        # the sweep's world frame shifts positions and map offsets by up to 1.3e5 px, so
        # the pixel-frame means agree to ~1e-11 px rather than bit for bit
        for prec, tol in ((cel.FP64, 1e-9), (cel.FP32, 1e-5)):
            tot, loc, g = Pf.elbo_grad(fld.theta, precision=prec)
            np.testing.assert_allclose(res[prec][1][rows], loc, rtol=tol)
            assert rel_l2(res[prec][2][rows], g) <= tol, (f, prec)
        Pf.close()
    assert np.isfinite(res[cel.FP64][0])
    assert rel(res[cel.FP32][0], res[cel.FP64][0]) <= 1e-5
