"""Staging arithmetic compiled for the host from the device headers: the double-float sum and
product keep ~48 bits, the continued fraction of DLMF 8.17.22 behind the binary64-polished
quantiles agrees with a long-double evaluation of the same recurrence to within its 1e-10
stopping rule, the certified tables err like the binary32 inversion they are checked against, and
the start tables of the Newton-Halley inversion estimate the root to within the 3e-4 that lets one
Halley step end it.  The host check of a host-resident YET's timestamps
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


# (mean, sd, max): sd above the largest a beta distribution with mean/max allows, so paper §3.3's
# clamp applies and alpha, beta come out near 1e-6
CLAMPED = [(1.0, 1.0, 1.5), (1000.0, 1500.0, 2000.0), (5e5, 9e5, 1.1e6), (1.0, 1.5, 2.5),
           (3e5, 6e5, 4e5)]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_clamped_records_invert_to_a_valid_quantile(oracle):
    """On clamped records the quantile is a near-step function: all but a few 1e-5 of the uniform
    grid maps to x within 1e-5 of 0 or 1, and in the narrow band between, x is extremely sensitive
    to the binary32 evaluation of I_x.  Every inversion must converge (no iteration cap), agree
    with the FP64 oracle within 1e-5 wherever the problem is well conditioned, and elsewhere be
    the exact quantile of a uniform within 5e-6 of u (backward error), checked by the oracle's
    I_x in binary64."""
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "clamp_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "clamp_check.cpp")], check=True)
        for mean, sd, mx in CLAMPED:
            rc, a_o, b_o = oracle.beta_moments(mean, sd, mx)
            assert rc == 1  # the oracle clamps too
            out = subprocess.run([exe, repr(mean), repr(sd), repr(mx), "509"], check=True,
                                 capture_output=True, text=True).stdout.splitlines()
            a, b, _ = out[0].split()
            a, b = float(a), float(b)
            assert a == pytest.approx(a_o, rel=1e-12) and b == pytest.approx(b_o, rel=1e-12)
            assert a < 2e-6 and b < 2e-6
            rows = [line.split() for line in out[1:]]
            assert len(rows) == 16_481 + 6_001
            n_sensitive = 0
            for u_s, xn_s, xs_s, cn, cs in rows:
                assert cn == "1" and cs == "1", (mean, u_s)
                u = float(u_s)
                xo, st = oracle.betaincinv(a, b, u)
                assert st == 0
                for x in (float(xn_s), float(xs_s)):
                    assert 0.0 <= x <= 1.0
                    if abs(x - xo) <= 1e-5:
                        continue
                    n_sensitive += 1
                    assert abs(oracle.betainc(a, b, x) - u) <= 5e-6, (mean, u, x, xo)
            assert 0 < n_sensitive <= 400  # the window holds the band, a few 1e-5 of u


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_binary32_tables_against_polished_quantiles():
    """The tables a run builds (binary32 knots, checked against the binary32 inversion) certify
    every record of the ELT value law and err like that inversion: over records staged as
    ara_add_elt stages them, x against the binary64-polished quantile, relatively, down to
    x = 1e-12."""
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "table_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "table_check.cpp")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    n_rec, certified = int(out[0]), int(out[1])
    worst_t, mean_t, worst_n, mean_n, worst_t4, worst_n4 = (float(v) for v in out[2:])
    assert n_rec == 1500 and certified == n_rec
    # the check admits 1e-6 in L plus the inversion's own rounding (capped at 1e-5) and 4 units
    # of the binary32 rounding of L (which dominates for tiny x); on average the tables sit within
    # a few 1e-7 of the exact quantile, as the inversion does
    assert worst_t <= 2.5e-5 and mean_t <= 1e-6
    assert worst_n <= 1e-5 and mean_n <= 5e-7
    # where losses matter (x >= 1e-4), both within 1e-5
    assert worst_t4 <= 1e-5 and worst_n4 <= 1e-5


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_staging_lngamma_against_the_c_library():
    """The staging's branch-free ln Gamma (shift by 8, Stirling's series through B_12) agrees with
    lgamma to ~1e-14 of max(1, |ln Gamma|), and ln B(a, b) over the ELT value law to 1e-12: far
    below the binary32 rounding of the constants it feeds."""
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "lngamma_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "lngamma_check.cpp")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    worst, worst_b = float(out[0]), float(out[1])
    assert worst <= 5e-14
    assert worst_b <= 1e-12
