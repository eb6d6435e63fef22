"""Host checks of the block fixed-point helpers of the mixed-form residual
(csrc/fx.cuh): the FP64 -> 64-bit integer conversion in a tile's unit, the
exact 128-bit coefficient product window, and the FP32 output of the
alpha-scaled residual (Step 1's scaling, Eq. 2.8) against exact 128-bit
integer and long double arithmetic.  The helpers are __host__ __device__;
this compiles their host form with the system C++ compiler."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2304_14021_gb300", "csrc")


@pytest.fixture(scope="module")
def fx_check(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fx") / "fx_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "fx_host", "fx_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe, "300000"], check=True, capture_output=True, text=True).stdout
    return {ln.split()[0]: ln.split()[1:] for ln in out.splitlines()}


@pytest.mark.parametrize("name", ["from_f64", "mul_shr", "to_f32_pair"])
def test_fx_helper_exact_or_bounded(fx_check, name):
    checked, failures, worst = fx_check[name]
    assert int(checked) > 0
    assert int(failures) == 0, (name, failures, worst)
