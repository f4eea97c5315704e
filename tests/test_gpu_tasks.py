"""Region task stages on the GPU (celeste_fit_tasks, the tasks side by side in one
sweep schedule): the same as fitting each task from the stage's starting parameters and
merging (bit for bit, a fixed number of sweeps), in both precisions, and against the
oracle's stage of task fits on the same tasks (FP64: positions 1e-3 px and fluxes 1e-4
relative, the fit targets, and the total ELBO 1e-8)."""
import numpy as np
import pytest

from oracle import tasks as OT
from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth
from tests.test_gpu_fit import rflux
from tests.test_tasks import _work

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste
    celeste.load()
    return celeste


def _crowded_tasks(cel, prob, parts=4, shift=None):
    work = _work(prob)
    t, n = cel.make_tasks(prob.theta[:, 0:2], work, work.sum() / parts, shift)
    assert n >= 2
    return t


@pytest.mark.parametrize("fp32", [False, True])
def test_fit_tasks_is_per_task_fits_merged(cel, fp32):
    """Overlapping tasks of the crowded region (their border sources share pixels), the
    stage against each task's own fit: FP64, and FP32 sweeps with the FP64 polish (the
    stage-start terms are taken in each phase's precision)."""
    prob = synth.config(2)
    task_of = _crowded_tasks(cel, prob)
    task_of[::7] = -1   # a few sources stay fixed
    P = cel.Problem(prob)
    kw = dict(precision=cel.FP32 if fp32 else cel.FP64, max_sweeps=2, sweep_tol=0.0)
    th, it, st, el = P.fit_tasks(prob.theta, task_of, **kw)
    ref = prob.theta.copy()
    for k in range(task_of.max() + 1):
        m = np.flatnonzero(task_of == k).astype(np.int32)
        tk, ik, _, _ = P.fit(prob.theta, which=m, **kw)
        ref[m] = tk[m]
        np.testing.assert_array_equal(it[m], ik[m])
    np.testing.assert_array_equal(th, ref)
    np.testing.assert_array_equal(th[task_of == -1], prob.theta[task_of == -1])
    assert el == P.elbo(ref, precision=cel.FP64)[0]
    P.close()


def test_fit_tasks_matches_oracle(cel):
    """Tasks over an independent set of the crowded region (the other sources fixed):
    each source's block solve is then independent of the path, so the stage matches the
    oracle's at the fit targets after one sweep."""
    from tests.test_gpu_fit import independent_set
    prob = synth.config(2)
    moving = independent_set(prob, 10)
    task_of = _crowded_tasks(cel, prob, shift=(20.0, -12.0))
    fixed = np.setdiff1d(np.arange(prob.n_src), moving)
    task_of[fixed] = -1
    assert len(np.unique(task_of[moving])) >= 2
    orc = Oracle(prob)
    o_th, _, _ = OT.fit_stage(orc, prob.theta, task_of, max_sweeps=1)
    o_el, _ = orc.elbo(o_th)
    P = cel.Problem(prob)
    th, _, st, el = P.fit_tasks(prob.theta, task_of, precision=cel.FP64, max_sweeps=1)
    for s in moving:
        assert np.abs(th[s, 0:2] - o_th[s, 0:2]).max() <= 1e-3, (s, th[s, :2], o_th[s, :2])
        assert abs(rflux(th[s]) / rflux(o_th[s]) - 1) <= 1e-4, s
    np.testing.assert_array_equal(th[fixed], prob.theta[fixed])
    assert abs(el - o_el) <= 1e-8 * abs(o_el)
    with pytest.raises(cel.CelesteError):
        bad = task_of.copy()
        bad[0] = -2
        P.fit_tasks(prob.theta, bad)
    P.close()
