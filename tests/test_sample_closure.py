"""The sampling argument the full-size GPU parity tests rest on, checked on the oracle
alone: a source's local objective depends only on the pixels of its patches, where E
and Var are sums over the sources whose patches cover them (the source and its
neighbours), so the sub-problem made of a sample and its neighbours gives the sampled
sources' local objectives and gradients of the full problem."""
import numpy as np

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests.helpers import neighbour_closure


def test_neighbour_closure_is_exact():
    prob = synth.config(2)
    sample = np.array([3, 17, 40], np.int64)
    keep = neighbour_closure(prob, sample)
    assert len(keep) < prob.n_src    # a real sub-problem
    sub = synth.subset(prob, keep)
    pos = np.searchsorted(keep, sample).astype(np.int32)
    full_l, full_g, _ = Oracle(prob).derivs(prob.theta, which=sample.astype(np.int32))
    sub_l, sub_g, _ = Oracle(sub).derivs(sub.theta, which=pos)
    assert np.max(np.abs(sub_l - full_l) / np.abs(full_l)) <= 1e-13
    assert np.linalg.norm(sub_g - full_g) <= 1e-12 * np.linalg.norm(full_g)


def test_non_neighbour_changes_nothing():
    """Moving a source that is not a neighbour leaves a sampled source's local
    objective unchanged (the sample's patches see no light of it)."""
    prob = synth.config(2)
    s = 3
    nb = set(int(o) for o in prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]])
    far = next(o for o in range(prob.n_src) if o != s and o not in nb)
    th2 = prob.theta.copy()
    th2[far, 0] += 0.7
    orc = Oracle(prob)
    a, _, _ = orc.derivs(prob.theta, which=np.array([s], np.int32))
    b, _, _ = orc.derivs(th2, which=np.array([s], np.int32))
    assert a[0] == b[0]
