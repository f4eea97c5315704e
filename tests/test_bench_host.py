"""Host logic of bench.py that needs no GPU: the clock-sample summary that decides
whether a timed run is kept, the Hessian leg's summary from its timings, and the
reference arm's JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _clocks(out):
    import bench
    c = bench.Clocks(0)
    c.out = out
    return c.summary()


def test_clock_summary_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _clocks("\n".join(rows) + "\n")
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    hot = rows + ["0, 1500, 2070, 1400.0, 0x48, Active, Active, Not Active, Active"]
    s = _clocks("\n".join(hot))
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]


def test_hessian_summary_from_timings():
    """The one-field workload's counts (3 PSF components, 8 + 6 profile components):
    FLOP per source-pixel, rates, the evaluation's and the Hessian pass's fractions of
    the FP32 peak, and no kernel entry when the pass's stage is missing."""
    import bench
    assert bench.hess_pass_flops_per_source_pixel(3, 8, 6) == 3 * (373 + 75 * 14) + 600
    assert bench.hess_flops_per_source_pixel(3, 8, 6) == 3 * (13 + 8 * 14) + 30 + 4869
    n_sp = 1_001_730
    stages = {"prep": 16.0, "contrib": 29.0, "gather": 9.0, "hess_adjoint": 199.0, "finalize": 123.0}
    h = bench.hessian_summary(n_sp, 1, 3, 8, 6, 0.373, 13.47, stages, 1.5e10)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert abs(h["value"] - n_sp / 0.373e-3) < 1.0
    assert abs(h["cost_vs_elbo_grad"] - 1.5e10 / h["value"]) < 1e-9
    r = h["roofline"]
    assert abs(r["achieved"] - 5274 * n_sp / 0.373e-3 / 1e12) < 1e-9 and abs(r["frac"] - r["achieved"] / peak) < 1e-12
    k = r["kernel"]
    assert k["name"] == "k_hess<float>" and k["flop_per_source_pixel"] == 4869
    assert abs(k["achieved"] - 4869 * n_sp / 199e-6 / 1e12) < 1e-9 and 0.29 < k["frac"] < 0.31
    assert abs(r["fp64"]["achieved"] - 7071 * n_sp / 13.47e-3 / 1e12) < 1e-9
    # two replicas: the rate doubles, each kernel's own rate does not
    h2 = bench.hessian_summary(n_sp, 2, 3, 8, 6, 0.373, 13.47, stages, 3.0e10)
    assert abs(h2["value"] - 2 * h["value"]) < 1.0 and h2["roofline"]["kernel"]["achieved"] == k["achieved"]
    assert abs(h2["roofline"]["frac"] - r["frac"]) < 1e-12
    assert bench.hessian_summary(n_sp, 1, 3, 8, 6, 0.373, 13.47, {}, 1.5e10)["roofline"]["kernel"] is None
    json.dumps(h)


def test_clock_summary_without_samples():
    assert _clocks("")["reasons"] == ["unsampled"]
    # a malformed line (too few fields) is not a sample
    assert _clocks("0, 2070\n")["reasons"] == ["unsampled"]
    # an unreadable clock field is skipped, the row still counts for its reasons
    s = _clocks("0, [N/A], [N/A], 0, 0x0, Not Active, Not Active, Active, Not Active\n")
    assert s["sm_mhz"] is None and s["reasons"] == ["sw_thermal_slowdown"]


def test_reference_arm_line():
    """`bench.py --impl reference` prints one JSON line whose value, e2e and
    cpu_baseline agree, in the metric and unit of the GPU arm."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "ELBO+grad source-pixel evals/s"
    assert d["unit"] == "source-pixel evals/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["dtype"] == "f64"
    assert d["value"] > 0
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "field_500src_5x2048x1489"
    assert d["config"]["source_pixels"] == 1001730
    # the GPU arm's config keys, so that the two lines name the same workload the same way
    assert {"workload", "sources", "source_pixels", "images", "image", "precision", "l2", "tuning",
            "parallelism"} <= set(d["config"])
    assert d["config"]["images"] == 5 and d["config"]["image"] == "2048x1489"
    sp = d["ms_per_step"] / 1000.0 * d["value"]
    assert 1 <= sp <= d["config"]["source_pixels"] * 1.000001


def test_oracle_rate_on_one_core_restores_the_thread_count():
    import bench
    from oracle.oracle import num_threads
    from paper_1801_10277_gb300 import synth
    prob = synth.config(0)
    before = num_threads()
    rate, cores, reps, secs = bench.oracle_rate(prob, min_seconds=0.2, threads=1)
    assert cores == 1 and reps >= 1 and rate > 0
    assert num_threads() == before
    rate_all, cores_all, _, _ = bench.oracle_rate(prob, min_seconds=0.2)
    assert cores_all == before and rate_all > 0


def test_step_bound_of_the_one_field_model():
    """3 PSF components x (1 star + 6 exp + 8 dev) = 45 mixture components per
    source-pixel: the FP32 pipe at 152 SMs x 128 lanes x 2 x 2.07 GHz over the item
    kernel's 3 (67 + 19 x 14) + 114 = 1,113 FLOP binds before the ex2 unit at 152 x 16 x
    2.07 GHz over 45 exps; the other covering sources' values add 3 (21 + 5 x 14) + 32 =
    305 FLOP and 45 exps per (pixel, other source)."""
    import bench
    assert bench.items_flops_per_source_pixel(3, 6, 8) == 1113
    assert bench.other_eval_flops(3, 6, 8) == 305
    b = bench.step_bound(3, 6, 8, 1.0e10)
    assert abs(b["evals_per_s_fp32_pipe"] - 152 * 128 * 2 * 2.07e9 / 1113) < 1.0
    assert abs(b["evals_per_s_ex2"] - 152 * 16 * 2.07e9 / 45) < 1.0
    assert b["evals_per_s_bound"] == b["evals_per_s_fp32_pipe"]
    assert abs(b["frac"] - 1.0e10 / b["evals_per_s_bound"]) < 1e-15
    b2 = bench.step_bound(3, 6, 8, 1.0e10, 0.1)
    assert abs(b2["flop_per_source_pixel"] - (1113 + 0.1 * 305)) < 1e-9


def test_reference_arm_under_torchrun_prints_once():
    """Launched as a multi-GPU run launches it (torchrun, two ranks), the reference
    arm prints one JSON line, from rank 0, and every rank exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
