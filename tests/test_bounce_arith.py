"""The exact integer arithmetic that starts a secondary ray (csrc/
bounce_arith.cuh: snapped origin parameter, mirror direction, side constant),
built for the host from the same header the kernel includes, equals 128-bit
integer division on random and adversarial cases.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    path = tmp_path_factory.mktemp("arith") / "bounce_arith_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_2112_05570_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "bounce_arith_check.cpp"), "-o", str(path), "-lm"])
    return str(path)


def test_bounce_arithmetic_equals_int128(exe):
    out = subprocess.run([exe, "600000", "7"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    words = out.stdout.split()
    cases, mismatches = int(words[1]), int(words[3])
    assert mismatches == 0 and cases > 300_000


def test_round_div_sqrt_equals_decimal(exe):
    """round(n / sqrt(m)) (halves up), which turns a direction given in a hit
    edge's frame into grid units, equals a 100-digit decimal evaluation on
    random pairs, perfect squares with exact halves and values next to halves."""
    from decimal import Decimal, ROUND_FLOOR, getcontext

    getcontext().prec = 100
    out = subprocess.run([exe, "round", "40000", "9"], capture_output=True, text=True, check=True).stdout
    bad = 0
    for line in out.splitlines():
        n, m, q = (int(w) for w in line.split())
        want = int((Decimal(n) / Decimal(m).sqrt() + Decimal("0.5")).to_integral_value(rounding=ROUND_FLOOR))
        bad += want != q
    assert bad == 0 and len(out.splitlines()) == 40000
