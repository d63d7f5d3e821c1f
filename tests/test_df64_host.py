"""The double-float arithmetic of the certified ordering (df64.cuh), compiled
for the host with g++ against a stand-in for the few CUDA declarations it
uses, and checked against double-precision libm over 400,000 arguments per
function: exp (Cody-Waite reduction, 2^(j/32) table, Taylor series), log1p
(one Newton step) and the two per-sample entropy functions the certified
re-evaluation sums.  Bounds: 2e-14 relative error per unit of |x| for exp,
5e-14 absolute for the others (FP64 itself carries about 1e-16; the pairs
carry about 48 bits).  A wrong sign of a table entry's low part, a dropped
low part of ln2/32 or a wrong sign of the low part of 1/3! each exceed them
(3e-8, 3e-9 and 2.2e-14 against 1.3e-14 for the exponential as written)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "df64_host", "df64_check.cpp")
BOUNDS = {"exp": 2e-14, "log1p": 5e-14, "logcosh": 5e-14, "gauss": 5e-14}


def test_double_float_functions_against_libm(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "df64_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "tests", "c", "df64_host"),
                    "-I", os.path.join(ROOT, "paper_2409_05500_gb300", "csrc"),
                    SRC, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    errs = {}
    for line in out.strip().splitlines():
        name, err, arg = line.split()
        errs[name] = (float(err), float(arg))
    assert set(errs) == set(BOUNDS)
    for name, bound in BOUNDS.items():
        assert errs[name][0] <= bound, (name, errs[name])
