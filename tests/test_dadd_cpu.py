"""The integer-ALU binary64 adder (csrc/pw_dadd.cuh) against the host's own
IEEE 754 addition, bit for bit, on 6 M seeded operand pairs that reach every
branch (tests/dadd_check.cpp, compiled with the host compiler)."""
import os
import shutil
import subprocess

import pytest

from paper_2107_13500_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_adder_matches_ieee_addition(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "dadd_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", build.CSRC,
                    os.path.join(HERE, "dadd_check.cpp"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    words = out.stdout.split()
    cases, accepted, bad = (int(words[k]) for k in (1, 3, 5))
    assert cases >= 6_000_000 and accepted > cases // 2 and bad == 0
