"""The plan-time dense symmetric eigensolver (host code of the library, CPU).

It factors the coarsest level of a composite domain.  Checked on closed forms
(the 1-D and 2-D Dirichlet Laplacians' eigenvalues, a rank-one update of the
identity), on a random symmetric matrix, and for A Q = Q Lambda and Q^T Q = I;
the memoised variant the planner calls returns bit for bit what a fresh
factorisation returns.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("symeig") / "symeig_check")
    subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(HERE, "native", "symeig_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.strip().splitlines():
        name, *vals = line.split()
        rows[name] = vals
    return rows


@pytest.mark.parametrize("name", ["random60", "laplace1d", "laplace2d", "rank1", "diagonal", "one", "two"])
def test_eigendecomposition(results, name):
    res, orth, ev = results[name]
    assert res != "FAIL"
    assert float(res) <= 1e-13 and float(orth) <= 1e-13
    if float(ev) >= 0:
        assert float(ev) <= 1e-13


def test_memoised_factorisation_is_bitwise_the_fresh_one(results):
    # repeated inputs, interleaved others, an eviction, a one-ulp change
    assert results["cached"] == ["ok", "3"]
