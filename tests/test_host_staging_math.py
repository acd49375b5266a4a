"""Staging arithmetic compiled for the host from the device headers: the table build's
double-float sum and product keep ~48 bits, the continued fraction of DLMF 8.17.22 that polishes
every knot agrees with a long-double evaluation of the same recurrence to within its 1e-10
stopping rule, and the start tables of the Newton-Halley inversion estimate the root to within
the 3e-4 that lets one Halley step end it.  The host check of a host-resident YET's timestamps
(vectorised where the CPU has AVX2) flags exactly what the plain definition flags."""

import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1310_2274_b300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_double_float_and_continued_fraction():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "df_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "df_check.cpp")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    worst_add, worst_mul, worst_cf = (float(v) for v in out)
    assert worst_add <= 2.0 ** -44  # relative to |a| + |b|: a few units of the 48-bit pair
    assert worst_mul <= 2.0 ** -45
    assert worst_cf <= 1e-10


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_start_tables_estimate_the_root():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "start_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "start_check.cpp")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    worst, mean, n, nan = float(out[0]), float(out[1]), int(out[2]), int(out[3])
    assert n == 60_000 and nan == 0
    assert worst <= 3e-4 and mean <= 1e-5


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_host_timestamp_check():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "tscheck_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-x", "c++", "-o", exe,
                        os.path.join(CSRC, "ara_tscheck.cu"), "-x", "none",
                        os.path.join(HERE, "tscheck_check.cpp")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    cases, wrong, flagged = (int(v) for v in out)
    assert cases == 400 and wrong == 0
    assert 250 <= flagged <= 300  # three kinds in four plant a NaN or a decrease
