"""The library built with CELESTE_CHECK_BOUNDS (device-side bounds checks on the item
records, candidate and table offsets, the tile lists and patch clipping, recording
CELESTE_ERR_BOUNDS instead of trapping): on valid problems no check fires and every
result equals the normal build's.  The checked library runs in a child process (the
binding loads one library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1801_10277_gb300 import synth, celeste as cel
cel.load(build_if_missing=True)
out = {}
for cfg in (0, 2):
    prob = synth.config(cfg)
    P = cel.Problem(prob)
    for prec in (cel.FP32, cel.FP64):
        tot, loc, g = P.elbo_grad(prob.theta, precision=prec)
        out[f"c{cfg}p{prec}_tot"] = np.array([tot]); out[f"c{cfg}p{prec}_loc"] = loc; out[f"c{cfg}p{prec}_g"] = g
        assert P.device_status() == 0, (cfg, prec, P.device_status())
    loc, g, h = P.hess(prob.theta, precision=cel.FP64)
    out[f"c{cfg}_h"] = h
    th, it, st, el = P.fit(prob.theta, precision=cel.FP32, max_sweeps=1)
    out[f"c{cfg}_fit"] = th
    assert P.device_status() == 0, (cfg, "fit", P.device_status())
    P.close()
np.savez(sys.argv[2], **out)
"""


def _run(tmp_path, checked):
    env = dict(os.environ)
    env["CELESTE_CHECK_BOUNDS"] = "1" if checked else "0"
    path = str(tmp_path / ("checked.npz" if checked else "plain.npz"))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, path], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(path)


def test_checked_build_is_silent_and_equal_on_valid_problems(tmp_path):
    plain = _run(tmp_path, False)
    checked = _run(tmp_path, True)
    assert set(plain.files) == set(checked.files)
    for k in plain.files:
        np.testing.assert_allclose(checked[k], plain[k], rtol=1e-12, atol=0, err_msg=k)
