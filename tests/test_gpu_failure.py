"""Failure detection without a GPU fault: a bounded device-side wait that nothing
satisfies gives up and reports CELESTE_ERR_TIMEOUT through a status word, and the
context stays usable (an evaluation afterwards matches one before)."""
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


def test_bounded_wait_times_out_and_context_survives(cel):
    import time
    prob = synth.config(0)
    P = cel.Problem(prob)
    before = P.elbo_grad(prob.theta, precision=cel.FP32)
    t0 = time.perf_counter()
    assert cel.selftest_bounded_wait() == cel.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    after = P.elbo_grad(prob.theta, precision=cel.FP32)
    assert after[0] == before[0]
    np.testing.assert_array_equal(after[2], before[2])
    P.close()
