"""The exact integer arithmetic that starts a secondary ray (csrc/
bounce_arith.cuh: snapped origin parameter, mirror direction, side constant),
built for the host from the same header the kernel includes, equals 128-bit
integer division on random and adversarial cases.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounce_arithmetic_equals_int128(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "bounce_arith_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_2112_05570_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "bounce_arith_check.cpp"), "-o", str(exe), "-lm"])
    out = subprocess.run([str(exe), "600000", "7"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    words = out.stdout.split()
    cases, mismatches = int(words[1]), int(words[3])
    assert mismatches == 0 and cases > 300_000
