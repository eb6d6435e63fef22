"""Host checks of the integer maps of the Step 2 column pass in register
four-step form (csrc/colr_map.cuh, used by k_cols_dct_fdi_r): the even/odd
reordering of the DCT-II via one complex FFT, the tile's chunk layout (a
bijection, with bank-conflict-free copies and DFT-step accesses), the lanes'
DCT-pair partners (an involution pairing p with N - p) and the schedule of
the pair solve (every entry updated once, against its pair).  The maps are
__host__ __device__; this compiles their host form with the system C++
compiler."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2304_14021_gb300", "csrc")


@pytest.fixture(scope="module")
def colr_check(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("colr") / "colr_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "colr_host", "colr_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {ln.split()[0]: ln.split()[1:] for ln in out.splitlines()}


@pytest.mark.parametrize("name", ["dct_pos", "chunk_bijection", "copy_banks", "lanes_partner", "dft_banks",
                                  "pair_schedule"])
def test_column_map_property(colr_check, name):
    checked, failures = colr_check[name]
    assert int(checked) > 0
    assert int(failures) == 0, (name, failures)
