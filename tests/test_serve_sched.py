"""The serving form's admission policy on the host (no GPU).

serve_sched.h holds the policy free of CUDA; serve_sched_check.cpp drives
it with stand-in lanes and requests: random arrivals and completions over
random lane counts, memory budgets and SM caps, with every admission
checked against the rules restated there (small requests first and in
arrival order, the oldest large request passed over at most four times,
the SM cap and the memory budget, nothing admissible left waiting, every
request served), plus the one-lane run order that the GPU serving test
also checks.
"""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_admission_policy_invariants():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "serve_sched_check")
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Werror",
                               "-I", os.path.join(ROOT, "paper_2607_23187_b300", "csrc"),
                               os.path.join(ROOT, "tests", "serve_sched_check.cpp"), "-o", exe])
        r = subprocess.run([exe, "300"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("ok 300 runs")
