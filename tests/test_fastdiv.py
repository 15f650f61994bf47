"""Division by a run-time divisor through a precomputed reciprocal
(csrc/fastdiv.h), used by the library's kernels to split an entry index into
(row, column, mode): checked on the CPU against the integer division over
every index below 2^22 and in the top 2^22 of [0, 2^31) for the divisors that
occur (mode counts, row lengths, half rows), and over the multiples of every
divisor below 70,000 and their neighbours."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2609_07172_gb300", "csrc")


def test_fast_division_matches_integer_division(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "fastdiv_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I" + CSRC, os.path.join(HERE, "native", "fastdiv_check.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout
    assert int(out.stdout.split()[1]) > 10 ** 8
