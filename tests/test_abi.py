"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/pint.h declares; parameter validation and footprint queries need no
GPU (pint_create validates before any CUDA call)."""
import ctypes as C
import os
import re

import pytest

from paper_2304_14021_gb300 import build_lib, pint

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return pint.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pint_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"pint_create", "pint_solve", "pint_residual", "pint_destroy", "pint_precond_apply"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_sizes_match_header_layout(lib):
    # pint_problem: 5 ints (+4 pad), 3 doubles, 2 ints, 3 doubles, 3 ints (+4 pad)
    assert C.sizeof(pint.Problem) == 24 + 24 + 8 + 24 + 16 + 8
    assert C.sizeof(pint.Stats) == 16 + 3 * 8 + 256 * 8 + 16 + 8 + 8 + 8
    assert C.sizeof(pint.TuneEntry) == 16


def test_strerror(lib):
    assert pint.strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5):
        assert len(pint.strerror(code)) > 5
    assert "unknown" in pint.strerror(-99)


BAD = [dict(dim=3), dict(nx=1), dict(nt=48), dict(nt=1 << 21), dict(nt=2048, nx=63), dict(nt=1), dict(alpha=0.0), dict(alpha=1.0),
       dict(theta=0.7), dict(theta=0.5, equation="cahn_hilliard", eps=0.05), dict(tol=0.0), dict(max_iter=0), dict(max_iter=256), dict(precision=7),
       dict(T=-1.0), dict(equation=5), dict(bc=3), dict(n_windows=0), dict(nx=2000, bc="ss"),
       dict(equation="linear_ch", eps=0.0), dict(init_guess=3), dict(dim=2, ny=1), dict(tol_update=-1.0)]


@pytest.mark.parametrize("bad", BAD)
def test_create_rejects_invalid_parameters(lib, bad):
    kw = dict(equation="biharmonic", dim=1, nx=64, bc="ss", nt=32, T=0.01)
    kw.update(bad)
    if kw.get("dim") == 2 and "ny" not in kw:
        kw["ny"] = 8
    p = pint.make_problem(**kw)
    h = C.c_void_p()
    assert lib.pint_create(C.byref(p), None, C.byref(h)) == pint.PINT_EINVAL
    assert not h.value
    assert lib.pint_footprint(C.byref(p)) == pint.PINT_EINVAL


def test_footprint_accounts_for_workspace(lib):
    # 2-D 256^2, nt=128: s (4 B/DOF mixed) + half spectrum (65*65536 complex64) + small tables
    mixed = pint.footprint(equation="linear_ch", dim=2, nx=256, ny=256, bc="neumann", nt=128, eps=0.05,
                           beta=0.5, T=0.1, precision="mixed")
    fp64 = pint.footprint(equation="linear_ch", dim=2, nx=256, ny=256, bc="neumann", nt=128, eps=0.05,
                          beta=0.5, T=0.1, precision="fp64")
    dof = 128 * 65536
    assert 4 * dof + 65 * 65536 * 8 < mixed < 4 * dof + 65 * 65536 * 8 + 8 * 2**20
    assert 8 * dof + 65 * 65536 * 16 < fp64 < 8 * dof + 65 * 65536 * 16 + 8 * 2**20


def test_null_arguments_rejected(lib):
    assert lib.pint_solve(None, None, None, None) == pint.PINT_EINVAL
    assert lib.pint_residual(None, None, None, None, None) == pint.PINT_EINVAL
    assert lib.pint_precond_apply(None, C.c_double(0.0), None, None) == pint.PINT_EINVAL
    lib.pint_destroy(None)


def test_precision_policy_falls_back_to_fp64_when_too_stiff():
    # 2^-24 * dt * max|spectrum| > 1 (1-D biharmonic, 4096 cells, dt = 0.01/32):
    # the FP32 inner solves cannot be refined, the problem runs (and is sized) in FP64.
    stiff = dict(equation="biharmonic", dim=1, nx=4096, bc="neumann", T=0.01, nt=32, alpha=1e-2, tol=1e-8)
    assert pint.footprint(**stiff, precision="mixed_ff") == pint.footprint(**stiff, precision="fp64")
    assert pint.footprint(**stiff, precision="mixed") == pint.footprint(**stiff, precision="fp64")
    # 2-D linearized CH 256^2, N_t = 128, T = 0.1: about 0.03, FP32 inner solves kept
    mild = dict(equation="linear_ch", dim=2, nx=256, ny=256, bc="neumann", eps=0.05, beta=0.5, T=0.1, nt=128,
                alpha=1e-2, tol=1e-8)
    assert pint.footprint(**mild, precision="mixed") < pint.footprint(**mild, precision="fp64")
    # 2-D biharmonic 512^2, dt = 0.01/256: amp about 10, a float-float request runs as PINT_MIXED
    mid = dict(equation="biharmonic", dim=2, nx=512, ny=512, bc="neumann", T=0.01, nt=256, alpha=1e-2, tol=1e-8)
    assert pint.footprint(**mid, precision="mixed_ff") == pint.footprint(**mid, precision="mixed")
    assert pint.footprint(**mid, precision="mixed") < pint.footprint(**mid, precision="fp64")


def test_crank_nicolson_accepted_for_linear_equations(lib):
    # theta = 1/2 is accepted for the linear equations (its footprint adds the b_1 buffer)
    kw = dict(equation="linear_ch", dim=2, nx=64, ny=64, bc="neumann", eps=0.05, beta=0.5, T=0.01, nt=32,
              alpha=1e-2, tol=1e-8, precision="mixed_ff")
    assert pint.footprint(**kw, theta=0.5) == pint.footprint(**kw, theta=1.0) + 64 * 64 * 8


def test_long_time_axis_accepted_for_even_point_counts(lib):
    kw = dict(equation="linear_ch", dim=1, nx=64, bc="neumann", eps=0.05, beta=0.5, T=1.0, alpha=1e-2, tol=1e-8)
    for nt in (2048, 65536, 131072, 1 << 20):
        assert pint.footprint(**kw, nt=nt) > 0
