"""torch.autograd.Function around the ELBO: forward = ELBO, backward = the adjoint
kernel recomputing the mixture terms from the forward's maps."""
import numpy as np
import pytest

from paper_1801_10277_gb300 import synth

pytestmark = pytest.mark.gpu


def test_autograd_matches_elbo_grad():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import autograd, celeste as cel
    prob = synth.config(2)
    P = cel.Problem(prob)
    for prec in (cel.FP64, cel.FP32):
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        th = torch.tensor(prob.theta, dtype=torch.float64, device="cuda", requires_grad=True)
        out = autograd.elbo(th, P, prec)
        assert out.item() == tot, prec
        (2.0 * out).backward()
        np.testing.assert_array_equal(th.grad.cpu().numpy(), 2.0 * g)
        # an evaluation between forward and backward does not corrupt the gradient
        th2 = torch.tensor(prob.theta, dtype=torch.float64, device="cuda", requires_grad=True)
        out2 = autograd.elbo(th2, P, prec)
        other = prob.theta.copy()
        other[:, 0] += 0.3
        P.elbo(other, precision=prec)
        out2.backward()
        np.testing.assert_array_equal(th2.grad.cpu().numpy(), g)
    P.close()
