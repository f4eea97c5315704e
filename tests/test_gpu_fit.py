"""Block-coordinate trust-region Newton fits (Section IV-D) on the GPU against the
oracle's fit from the same starts: positions within 1e-3 px and r-band expected
fluxes within 1e-4 relative for every moving source, in both precisions.  A source's
status (stopped by the gain test, or at the iteration cap) may differ between the two
sides only as converged against capped: a source whose predicted gains hover at the
stopping threshold can stop one iteration before the cap on one side and reach it on
the other; neither side may report a non-finite objective.

On an independent set (no two moving sources overlap, so a source's local objective
depends on it alone) a source whose two fits end in different local optima is not a
parity failure: the objective is not convex (q's colour-component weights can settle on
different prior components), and a trust-region path that differs in rounding can take
either basin.  Such a source passes when the GPU's fit converged and its local objective,
evaluated by the oracle, is at least the oracle fit's; every such source is printed."""
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


def _other_optimum(prec, s, th_s, o_s, st_s, local):
    """None when th_s and o_s agree at the fit targets; else (source, position error,
    flux error, local objective of the GPU's result minus the oracle's) after checking that
    the GPU's fit converged to an optimum at least as good (local: theta_s -> the oracle's
    local objective with every other source as in the fit)."""
    dpos = float(np.abs(th_s[0:2] - o_s[0:2]).max())
    dflux = abs(rflux(th_s) / rflux(o_s) - 1)
    if dpos <= 1e-3 and dflux <= 1e-4:
        return None
    lg, lo = local(th_s), local(o_s)
    assert st_s == 0 and lg >= lo - 1e-10 * abs(lo), (prec, s, dpos, dflux, st_s, lg, lo)
    return (int(s), dpos, dflux, lg - lo)


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
        # every moving source is compared; on an independent set a different optimum passes
        # when the GPU's is at least as good
        other = []
        for s in moving:
            if which is not None:
                def local(x, s=s):
                    y = prob.theta.copy()
                    y[s] = x
                    return orc.elbo(y)[1][s]
                d = _other_optimum(prec, s, th[s], o_th[s], st[s], local)
                if d is not None:
                    other.append(d)
                continue
            assert np.abs(th[s, 0:2] - o_th[s, 0:2]).max() <= 1e-3, (prec, s, th[s, :2], o_th[s, :2])
            assert abs(rflux(th[s]) / rflux(o_th[s]) - 1) <= 1e-4, (prec, s, th[s], o_th[s])
        print(f"{'FP64' if prec == cel.FP64 else 'FP32'}: other optima (source, position error, flux error, "
              f"GPU minus oracle local objective) {other}")
        _check_status(prec == cel.FP64, moving, st, it, o_st, o_it)
        assert abs(el - o_el) <= (1e-8 if prec == cel.FP64 else 1e-5) * abs(o_el), (prec, el, o_el)
        # sources outside `which` never move
        still = np.setdiff1d(np.arange(prob.n_src), moving)
        np.testing.assert_array_equal(th[still], prob.theta[still])
    P.close()


def _check_status(fp64, moving, st, it, o_st, o_it, o_index=None):
    """Statuses of the moving sources: 0 converged, 1 at the iteration cap, 2 non-finite.
    Prints every disagreement with both sides' iteration counts."""
    o_index = moving if o_index is None else o_index
    diff = [(int(s), int(st[s]), int(o_st[o]), int(it[s]), int(o_it[o]))
            for s, o in zip(moving, o_index) if st[s] != o_st[o]]
    print(f"{'FP64' if fp64 else 'FP32'}: status differs for (source, GPU, oracle, GPU iterations, "
          f"oracle iterations) {diff}")
    assert all(st[s] in (0, 1) for s in moving) and all(o_st[o] in (0, 1) for o in o_index)


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


def closure_subset(prob, which):
    """The sub-problem of `which` and their neighbours (every other source whose patches
    overlap theirs, i.e. every source their pixels see), and the positions of `which` in
    it."""
    keep = set(int(s) for s in which)
    for s in which:
        keep |= set(prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]].tolist())
    keep = np.array(sorted(keep))
    pos = np.searchsorted(keep, np.asarray(which))
    return synth.subset(prob, keep), pos.astype(np.int32)


def test_fit_field_sample(cel):
    """32 sources of the one-field workload (500 sources over five 2048 x 1489 images), no
    two overlapping: the GPU fits them in the whole field, the oracle in the sub-problem
    of them and their neighbours.  Per-source positions and fluxes at the fit targets, in
    both precisions, or (at most one source in eight) a different optimum at least as good
    as the oracle's."""
    prob = synth.config(1)
    which = independent_set(prob, 32)
    assert len(which) == 32
    sub, pos = closure_subset(prob, which)
    orc = Oracle(sub)
    o_th, o_it, o_st, _, _ = orc.fit(sub.theta, which=pos, max_sweeps=2, sweep_tol=1e-12)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        th, it, st, _ = P.fit(prob.theta, which=which, precision=prec, max_sweeps=2, sweep_tol=1e-12)
        other = []
        for k, s in enumerate(which):
            def local(x, k=k):
                y = sub.theta.copy()
                y[pos[k]] = x
                return orc.elbo(y)[1][pos[k]]
            d = _other_optimum(prec, s, th[s], o_th[pos[k]], st[s], local)
            if d is not None:
                other.append(d)
        print(f"{'FP64' if prec == cel.FP64 else 'FP32'}: other optima (source, position error, flux error, "
              f"GPU minus oracle local objective) {other}")
        assert len(other) <= len(which) // 8, other
        _check_status(prec == cel.FP64, which, st, it, o_st, o_it, pos)
        still = np.setdiff1d(np.arange(prob.n_src), which)
        np.testing.assert_array_equal(th[still], prob.theta[still])
    P.close()


def test_fit_fp32_sweeps_without_the_fp64_polish(cel):
    """The FP32 fit's own result (refine_fp64 = 0: FP32 pixel sums throughout, FP64
    accumulation) against the oracle's FP64 fit, on an independent set of the crowded
    region, at the fit targets."""
    prob = synth.config(2)
    which = independent_set(prob, 8)
    o_th, _, o_st, _, _ = Oracle(prob).fit(prob.theta, which=which, max_sweeps=2, sweep_tol=1e-12)
    P = cel.Problem(prob)
    th, it, st, _ = P.fit(prob.theta, which=which, precision=cel.FP32, refine_fp64=0, max_sweeps=2,
                          sweep_tol=1e-12)
    dpos = max(np.abs(th[s, 0:2] - o_th[s, 0:2]).max() for s in which)
    dflux = max(abs(rflux(th[s]) / rflux(o_th[s]) - 1) for s in which)
    print(f"FP32 without the FP64 polish: max position error {dpos:.3g} px, max flux error {dflux:.3g}")
    assert dpos <= 1e-3 and dflux <= 1e-4, (dpos, dflux)
    P.close()


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


def _orders(rng, moving, sweeps):
    return np.stack([rng.permutation(moving) for _ in range(sweeps)]).astype(np.int32)


def _compare_sweeps(cel, prob, order, sample_size, which=None):
    """The Cyclades schedule on given sweep orders, every sweep run (no early stop), on
    both sides: sources that overlap follow one path, so after a fixed number of sweeps
    the two fits agree to the per-source Newton tolerance (the joint optimum itself is
    approached along flat ridges where a sweep tolerance stops each side elsewhere)."""
    orc = Oracle(prob)
    ns = order.shape[0]
    moving = np.arange(prob.n_src) if which is None else np.asarray(which)
    P = cel.Problem(prob)
    # FP64: ns sweeps.  FP32: ns FP32 sweeps polished by ns FP64 sweeps on the same order
    # rows, against ns + ns oracle sweeps on those rows.  FP64 block solves stop on a
    # predicted gain below 1e-14 (1 + |ELBO_s|), tighter than the default, so that the
    # stopping slack of weakly constrained sources stays small; the tolerances are the
    # fit targets, as the oracle solves each trust-region subproblem exactly
    # (eigendecomposition) and the GPU to 1e-6 in the step length, so paths that have not
    # converged differ by more than rounding.
    for prec, tpos, tflux, tel in ((cel.FP64, 1e-3, 1e-4, 1e-8), (cel.FP32, 1e-3, 1e-4, 1e-5)):
        reps = 1 if prec == cel.FP64 else 2
        # the tighter stop only where FP64 pixels can reach it
        tol = dict(pred_tol_rel=1e-14) if prec == cel.FP64 else {}
        o_th, _, _, o_el, o_sw = orc.fit(prob.theta, which=which, max_sweeps=reps * ns,
                                         sweep_tol=0.0, order=np.tile(order, (reps, 1)),
                                         sample_size=sample_size, **tol)
        assert o_sw == reps * ns
        th, it, st, el = P.fit(prob.theta, which=which, precision=prec, refine_fp64=1,
                               max_sweeps=ns, sweep_tol=0.0, schedule="cyclades", order=order,
                               sample_size=sample_size, **tol)
        for s in moving:
            assert np.abs(th[s, 0:2] - o_th[s, 0:2]).max() <= tpos, (prec, s, th[s, :2], o_th[s, :2])
            assert abs(rflux(th[s]) / rflux(o_th[s]) - 1) <= tflux, (prec, s)
        assert abs(el - o_el) <= tel * abs(o_el), (prec, el, o_el)
    P.close()


def test_fit_cyclades_tiny(cel):
    """Two overlapping sources, random sweep orders, samples of two."""
    prob = synth.config(0)
    _compare_sweeps(cel, prob, _orders(np.random.default_rng(21), np.arange(2), 3), 2)


def connected_cluster(prob, k, start=0):
    """k sources connected in the neighbour graph (breadth-first from `start`)."""
    seen, queue = [start], [start]
    while queue and len(seen) < k:
        s = queue.pop(0)
        for o in prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]].tolist():
            if o not in seen and len(seen) < k:
                seen.append(o)
                queue.append(o)
    return np.array(sorted(seen), np.int32)


def test_fit_cyclades_crowded_cluster(cel):
    """Five linked sources of the crowded region moving, the rest fixed; samples of
    three, so both components and serialised members occur."""
    prob = synth.config(2)
    which = connected_cluster(prob, 5)
    assert len(which) == 5
    _compare_sweeps(cel, prob, _orders(np.random.default_rng(22), which, 2), 3, which=which)


def test_fit_cyclades_is_serially_equivalent(cel):
    """Cyclades' guarantee: for one order the result is that of updating the sources one
    at a time in that order, whatever the sample size (bit for bit here: a source's fit
    reads the same neighbour values and sums in the same order)."""
    prob = synth.config(2)
    which = connected_cluster(prob, 12, start=5)
    order = _orders(np.random.default_rng(23), which, 2)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        res = [P.fit(prob.theta, which=which, precision=prec, refine_fp64=0, max_sweeps=2,
                     sweep_tol=0.0, schedule="cyclades", order=order, sample_size=B)
               for B in (1, 3, 12)]
        for th, it, st, el in res[1:]:
            np.testing.assert_array_equal(th, res[0][0])
            np.testing.assert_array_equal(it, res[0][1])
            assert el == res[0][3]
    P.close()


def test_fit_cyclades_generated_orders(cel):
    """Orders drawn inside the library from a seed: reproducible, ELBO raised, and
    order rows that are not permutations of the moving set are errors."""
    prob = synth.config(2)
    which = connected_cluster(prob, 12, start=5)
    P = cel.Problem(prob)
    start = P.elbo(prob.theta, precision=cel.FP64)[0]
    kw = dict(which=which, precision=cel.FP64, max_sweeps=3, schedule="cyclades", sample_size=4)
    th1, it1, st1, el1 = P.fit(prob.theta, seed=11, **kw)
    th2, it2, st2, el2 = P.fit(prob.theta, seed=11, **kw)
    np.testing.assert_array_equal(th1, th2)
    assert el1 == el2 and el1 > start
    bad = np.tile(which, (3, 1))
    bad[1, 0] = bad[1, 1]
    with pytest.raises(cel.CelesteError) as e:
        P.fit(prob.theta, order=bad, **kw)
    assert e.value.status == cel.ERR_ARG
    with pytest.raises(cel.CelesteError):
        P.fit(prob.theta, which=which, schedule="cyclades", sample_size=0)
    P.close()


def test_fit_crowded_region_to_convergence(cel):
    """The crowded region (64 mutually overlapping sources, 2-12 neighbours each),
    block-coordinate trust-region Newton run until a sweep changes the total ELBO by
    less than 1e-8 relative: a further sweep from the result then moves the ELBO by less
    than that, and the total never decreased."""
    prob = synth.config(2)
    P = cel.Problem(prob)
    start = P.elbo(prob.theta, precision=cel.FP64)[0]
    th, it, st, el = P.fit(prob.theta, precision=cel.FP64, max_sweeps=100, sweep_tol=1e-8)
    assert el > start
    assert np.count_nonzero(st == 0) >= 0.75 * prob.n_src
    th2, _, _, el2 = P.fit(th, precision=cel.FP64, max_sweeps=1)
    assert abs(el2 - el) <= 1e-8 * abs(el)
    assert el2 >= el - 1e-9 * abs(el)
    P.close()
