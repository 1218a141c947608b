"""The float64 log series' quotient on the device is computed by Markstein's
method (IBM J. Res. Dev. 34(1), 1990) rather than a division: an approximate
float reciprocal, two Newton steps, a reciprocal step on the exact residual,
and two quotient corrections.  Markstein's theorems make the result the
correctly rounded quotient when the reciprocal step starts within one ulp and
the divisor's significand is not all ones; the one such divisor in range,
2 - 2^-52, is set directly.  These tests restate the steps in C and check them
against the host's correctly rounded division on random and edge inputs of the
reduced range, with the initial reciprocal moved by several float ulps, and
that without the special case the all-ones divisor does differ.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path_factory.mktemp("quotient") / "quotient_check")
    subprocess.run([cc, "-O2", "-std=c99", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "quotient_check.c"),
                    "-lm"], check=True)
    return exe


def run(exe, *args):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True)
    return r.returncode, r.stdout


def test_quotient_is_correctly_rounded(checker):
    rc, out = run(checker, 400000, 4)
    assert rc == 0, out
    assert out.strip().endswith("0 differ")


def test_quotient_tolerates_a_coarse_reciprocal(checker):
    rc, out = run(checker, 20000, 2048)
    assert rc == 0, out


def test_all_ones_divisor_needs_the_special_case(checker):
    rc, out = run(checker, 0, 0, 1)
    assert rc == 1 and "0x1.ffffffffffffep-1" in out, out
