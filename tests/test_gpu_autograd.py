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


def test_gpu_derivatives_match_central_differences():
    """The GPU gradient and per-source Hessian (FP64 pixels) against central differences
    of the GPU itself, h = 1e-6: on the crowded region, for three sources and a sample of
    coordinates covering position, shape, brightness, colour, type and the colour-class
    weights.  A source's local objective depends on its own parameters exactly as the total
    does (pixels outside its patches do not), so its difference quotient is taken on the
    local objective (smaller, so the quotient's rounding error is smaller); the Hessian's
    columns are difference quotients of the FP64 gradient."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10277_gb300 import celeste as cel
    prob = synth.config(2)
    P = cel.Problem(prob)
    th0 = prob.theta.copy()
    loc0, g0, hs = P.hess(th0, precision=cel.FP64)
    h = 1e-6
    coords = [0, 1, synth.I_EDEV, synth.I_AXIS, synth.I_ANGLE, synth.I_SCALE, synth.I_R1, synth.I_R2 + 1,
              synth.I_C1 + 2, synth.I_C2 + 5, synth.I_A, synth.I_K + 3, synth.I_K + 12]
    worst_g = worst_h = 0.0
    for s in (0, prob.n_src // 2, prob.n_src - 1):
        for j in coords:
            tp, tm = th0.copy(), th0.copy()
            tp[s, j] += h
            tm[s, j] -= h
            _, lp, gp = P.elbo_grad(tp, precision=cel.FP64)
            _, lm, gm = P.elbo_grad(tm, precision=cel.FP64)
            fd = (lp[s] - lm[s]) / (2 * h)
            # the quotient's rounding error: a few ulps of the local objective over 2h
            tol = 1e-6 * abs(g0[s, j]) + 64 * np.finfo(float).eps * abs(loc0[s]) / (2 * h) + 1e-7
            err = abs(fd - g0[s, j])
            worst_g = max(worst_g, err / tol)
            assert err <= tol, (s, j, fd, g0[s, j])
            col = (gp[s] - gm[s]) / (2 * h)
            scale = np.abs(hs[s]).max()
            errh = np.abs(col - hs[s][:, j]).max()
            worst_h = max(worst_h, errh / scale)
            assert errh <= 1e-5 * scale, (s, j, errh, scale)
    print(f"worst gradient error / tolerance {worst_g:.3g}, worst Hessian column error / max |H| {worst_h:.3g}")
    P.close()
