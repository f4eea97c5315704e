"""The FP32 Hessian kernel's galaxy terms, evaluated in the frame that whitens each PSF
component (Section IV-D's exact second derivatives, reorganised as 35 weighted sums per
component), run on the host against the pixel-frame formulas in FP64.  The whitened
evaluation must be as accurate as the pixel-frame formulas evaluated in FP32 (at most
twice their worst error, and within 3e-4 of each quantity's scale); a dropped term, a
wrong index or a transposed map gives errors of order one."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1801_10277_gb300", "csrc")


def test_whitened_frame_matches_pixel_frame(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "whitened_frame_check")
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=compute_103a",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, os.path.join(HERE, "whitened_frame_check.cu"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    rows = {}
    for line in r.stdout.split("\n"):
        parts = line.split()
        if len(parts) == 3:
            rows[parts[0]] = (float(parts[1]), float(parts[2]))
    assert set(rows) == {"value", "gradient", "e_dev", "hessian", "e_dev_gradient"}, r.stdout
    for name, (whitened, pixel32) in rows.items():
        assert whitened <= 3e-4, (name, whitened)
        assert whitened <= 2.0 * pixel32 + 1e-6, (name, whitened, pixel32)
