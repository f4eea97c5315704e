"""GPU parity on the two large workloads, at full size, through the C ABI.

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
