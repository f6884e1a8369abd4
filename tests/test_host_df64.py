"""Host check of the double-float (df64) bit-level conversions that the FP32-pipe
refinement residuals, SpMM and Krylov basis rely on: compiled from tests/df64_check.cpp."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_df64_split_and_widen_are_exact():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "df64_check")
        subprocess.run([gxx, "-O2", "-std=c++17", os.path.join(HERE, "df64_check.cpp"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
