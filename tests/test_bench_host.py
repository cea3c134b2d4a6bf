"""bench.py pieces that run on the host: the reference arm (the oracle timed
on a bounded sample of the workload) reports a positive rate on a lattice
smaller than its per-step sample, and the recorded-profile reader."""
import json
import subprocess
import sys
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_on_a_small_lattice():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "bcc16_k4", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["value"] == line["value"] and 1 <= cb["cores"] <= cb["host"]["nproc"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_recorded_profile_matches_kernel_source():
    sys.path.insert(0, ROOT)
    import bench
    n = 1070774656
    rec = bench._recorded_profile(n)
    # the committed ncu summary was taken on the current tiled-kernel source;
    # its DRAM bytes scale with the sites from the profiled lattice
    assert rec is not None and rec["dram_bytes_per_launch"] > 0
    assert rec["dram_bytes_per_launch"] == bench._recorded_profile(rec["profiled_sites"])[
        "dram_bytes_per_launch"] * n // rec["profiled_sites"]
    lim = rec["limiter"]
    assert 0 < lim["shared_pipe_frac"] <= 1 and 0 < lim["issue_active_frac"] <= 1


def test_local_model_cpu_baseline(orc):
    """The --mode local line's CPU baseline: the oracle's local sweeps on a
    bounded lattice of the workload's recipe."""
    import bench
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("bcc812_k5")
    cb = bench.cpu_baseline_local(w, 3, 1.0)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert "lattice" in cb["sample"]
