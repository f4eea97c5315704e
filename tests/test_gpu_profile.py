"""Per-stage timing: the concurrent (mode 1) and serialised (mode 2) profiling runs give
the same bits as an unprofiled call, report the same stages, and bad modes are
rejected."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("cfg", [0, 2])
def test_profiled_runs_match_and_report_the_stages(cel, cfg):
    prob = synth.config(cfg)
    P = cel.Problem(prob)
    ref = P.elbo_grad(prob.theta, precision=cel.FP32)
    stages = {}
    for serial in (False, True):
        P.profile(True, serial=serial)
        got = P.elbo_grad(prob.theta, precision=cel.FP32)
        stages[serial] = P.profile_read()
        P.profile(False)
        assert got[0] == ref[0]
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_array_equal(got[2], ref[2])
    assert set(stages[False]) == set(stages[True])
    assert {"items"} <= set(stages[True])
    for v in stages[True].values():
        assert v[0] > 0 and v[1] >= 1
    with pytest.raises(cel.CelesteError) as e:
        cel._check(P.L.celeste_profile_enable(P.h, 3))
    assert e.value.status == cel.ERR_ARG
    P.close()
