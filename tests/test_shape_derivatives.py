"""The Hessian epilogue's galaxy-shape derivatives (the world-frame ellipse's first and
second derivatives over axis ratio, angle and scale, mapped through each patch's A) run
on the host against central differences of G = A W A' with W written as
sigma^2 R(phi) diag(1, rho^2) R(phi)' (Section III's galaxy shape)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1801_10277_gb300", "csrc")


def test_shape_derivatives_match_central_differences(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "shape_derivs_check")
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=compute_103a",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, os.path.join(HERE, "shape_derivs_check.cu"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    worst = dict((p[0], float(p[1])) for p in (ln.split() for ln in r.stdout.split("\n")) if len(p) == 2)
    # central-difference error: ~1e-10 (first, h = 1e-6), ~1e-8 (second, h = 1e-4)
    assert worst["first"] <= 1e-8, worst
    assert worst["second"] <= 1e-6, worst
