"""The block fixed-point residual of PINT_MIXED (integer pipes; linear equations
and the Cahn-Hilliard u^3 term) against the oracle's FP64 residual (Eq. 2.6 /
Eq. 4.8 with alpha = 0) and the FP64 residual kernel,
element by element, through the C ABI.

On a random iterate the residual is of the size of its terms, and both GPU
forms must match the oracle to 1e-13 of max|r| at every point, boundary rows
and ragged tiles included.  At the sequential solution the residual is pure
rounding: there every form must stay within a few FP64 units of the terms'
scale (an FP32-accurate residual would be 1e-7 of it).
"""
import numpy as np
import pytest

from oracle import pint_oracle as O
from paper_2304_14021_gb300 import build_lib, pint, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def full(kw):
    d = dict(equation="biharmonic", dim=1, nx=64, ny=1, bc="ss", eps=1.0, beta=0.0, T=0.01, nt=32, n_windows=1,
             theta=1.0, alpha=1e-2, tol=1e-12, max_iter=100, precision="mixed", init_guess=0)
    d.update(kw)
    if d["dim"] == 1:
        d["ny"] = 1
    return d


def oprob(kw):
    keys = ("equation", "dim", "nx", "ny", "bc", "eps", "beta", "T", "nt", "n_windows", "theta", "alpha")
    return O.Problem(**{k: kw[k] for k in keys if k in kw})


CASES = [
    dict(equation="biharmonic", dim=1, nx=64, bc="ss", nt=32, T=0.01),                                  # config 1 shape
    dict(equation="linear_ch", dim=2, nx=256, ny=256, bc="neumann", nt=8, T=0.1 * 8 / 128, eps=0.05, beta=0.5),
    dict(equation="linear_ch", dim=2, nx=48, ny=48, bc="neumann", nt=4, T=5e-3, eps=0.05, beta=0.5),    # ragged tiles
    dict(equation="biharmonic", dim=2, nx=40, ny=40, bc="ss", nt=8, T=1e-3),                            # odd reflections
    dict(equation="linear_ch", dim=2, nx=33, ny=33, bc="neumann_v", nt=4, T=1e-3, eps=0.05, beta=0.4),  # vertex grid
    dict(equation="linear_ch", dim=1, nx=700, bc="neumann", nt=8, T=1e-4, eps=0.05, beta=-0.5),         # signed beta^2
    dict(equation="linear_ch", dim=2, nx=64, ny=64, bc="neumann", nt=8, T=0.01, eps=0.05, beta=0.5, theta=0.5),
    dict(equation="biharmonic", dim=1, nx=1000, bc="neumann", nt=4, T=1e-6, theta=0.5),                 # CN, 1-D
    dict(equation="linear_ch", dim=1, nx=5, bc="ss", nt=2, T=1e-3, eps=0.1, beta=0.3),                  # tiny
    dict(equation="linear_ch", dim=1, nx=32, bc="neumann", nt=8, T=1e-3, eps=0.01, beta=0.57),          # c1 > c2
    dict(equation="cahn_hilliard", dim=2, nx=64, ny=64, bc="neumann", nt=8, T=8e-4, eps=0.05),          # u^3 term
    dict(equation="cahn_hilliard", dim=1, nx=130, bc="neumann", nt=4, T=1e-4, eps=0.05),                # ragged
    dict(equation="cahn_hilliard", dim=2, nx=40, ny=40, bc="ss", nt=4, T=1e-4, eps=0.1),                # odd reflections
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fx_residual_matches_oracle_and_fp64_kernel_on_random_iterates(case):
    kw = full(CASES[case])
    p = oprob(kw)
    u0 = synth.u0_uniform(p.nspace, -1, 1, 10 + case)
    U = synth.random_iterate(p.nt, p.nspace, 20 + case)
    ref = O.residual(p, u0, U)
    out = {}
    for prec in ("mixed", "fp64"):
        with pint.Solver(**dict(kw, precision=prec)) as s:
            if prec == "mixed":
                s.set_fx_residual(True)   # raises where the fixed-point form is not supported
            r = torch.empty(p.nt, p.nspace, dtype=torch.float64, device="cuda")
            rel = s.residual(dev(u0), dev(U), r)
            out[prec] = (host(r), rel)
    scale = np.max(np.abs(ref))
    for prec, (r, rel) in out.items():
        assert np.max(np.abs(r - ref)) <= 1e-13 * scale, (prec, np.max(np.abs(r - ref)) / scale)
        assert abs(rel - np.linalg.norm(ref) / O.rhs_norm(p, u0)) <= 1e-12 * rel
    assert np.max(np.abs(out["mixed"][0] - out["fp64"][0])) <= 1e-13 * scale


@pytest.mark.parametrize("case", [0, 2, 3, 4, 6, 7, 9])
def test_fx_residual_at_the_sequential_solution_is_fp64_rounding(case):
    # At the sequential solution r = b - K(U) vanishes up to rounding.  The sums that
    # form it reach max|u| (1/dt + ||A||_inf) (the stencil terms, before they cancel):
    # every form must resolve r to about a hundred FP64 units of that scale (an
    # FP32-accurate residual would leave ~1e-8 of it).
    kw = full(CASES[case])
    p = oprob(kw)
    u0 = synth.u0_uniform(p.nspace, -1, 1, 30 + case)
    U = O.sequential(p, u0)[-p.nt:]
    ref = O.residual(p, u0, U)
    a_inf = np.max(np.asarray(abs(O.operator_A(p)).sum(axis=1)))
    scale = np.max(np.abs(U)) * (1.0 / p.dt + a_inf)
    errs = {}
    for prec in ("mixed", "fp64"):
        with pint.Solver(**dict(kw, precision=prec)) as s:
            if prec == "mixed":
                s.set_fx_residual(True)
            r = torch.empty(p.nt, p.nspace, dtype=torch.float64, device="cuda")
            s.residual(dev(u0), dev(U), r)
            errs[prec] = np.max(np.abs(host(r) - ref)) / scale
    assert errs["mixed"] < 1e-14, errs
    assert errs["fp64"] < 1e-14, errs
    # and no worse than the FP64 kernel itself (both measured against the oracle's own rounding)
    assert errs["mixed"] <= 2.0 * errs["fp64"] + 1e-17, errs


@pytest.mark.parametrize("nx", [512, 1024])
def test_fx_residual_stiff_smooth_problem_converges_like_fp64(nx):
    # 1-D biharmonic, Neumann, T = 0.01 over 16 steps: dt ||A|| ~ 1e9-1e10 (PINT_MIXED by the precision
    # policy).  The solution is smooth, so the residual's terms are far below their worst-case bounds:
    # the fixed-point residual must resolve them relative to their actual size, as FP64 does, or the
    # iteration stalls above its rounding floor.
    kw = full(dict(equation="biharmonic", dim=1, nx=nx, bc="neumann", nt=16, T=0.01, tol=1e-10, tol_update=1e-9,
                   init_guess=2, max_iter=60))
    p = oprob(kw)
    x = (np.arange(nx) + 0.5) / nx
    u0 = np.cos(np.pi * x) + 0.5 * np.cos(3 * np.pi * x) - 0.25 * np.cos(7 * np.pi * x)
    res = {}
    for fx in (True, False):
        with pint.Solver(**kw) as s:
            s.set_fx_residual(fx)
            U = torch.zeros(p.nt, p.nspace, dtype=torch.float64, device="cuda")
            st = s.solve(dev(u0), U, check=False)
            res[fx] = (host(U), st)
    st_fx, st_64 = res[True][1], res[False][1]
    assert st_fx["rc"] == 0 and st_64["rc"] == 0, (st_fx, st_64)
    assert st_fx["iters"] <= st_64["iters"] + 2, (st_fx["hist"], st_64["hist"])
    assert O.rel_err(res[True][0], res[False][0]) < 1e-8


@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
def test_mixed_fx_solve_reaches_fp64_floor(alpha):
    # 2-D linearized CH 64^2 (config 2's parameters): PINT_MIXED with the fixed-point
    # residual refines the complex64 inner solves to rho <= 1e-12 and the sequential
    # solution to 1e-10, which an FP32-accurate residual could not reach.
    kw = full(dict(equation="linear_ch", dim=2, nx=64, ny=64, bc="neumann", eps=0.05, beta=0.5, nt=32,
                   T=32 * 0.1 / 128, alpha=alpha, tol=1e-12, init_guess=2))
    p = oprob(kw)
    u0 = synth.u0_uniform(p.nspace, -0.05, 0.05, 0)
    with pint.Solver(**kw) as s:
        U = torch.zeros(p.nt, p.nspace, dtype=torch.float64, device="cuda")
        st = s.solve(dev(u0), U, check=False)
        U = host(U)
    assert st["rc"] == 0 and st["precision"] == "mixed", st
    assert O.rel_err(U, O.sequential(p, u0)) < 1e-10


@pytest.mark.parametrize("case", [1, 6])
def test_mixed_solve_same_with_fx_and_fp64_residual(case):
    # The same solve with the fixed-point residual and with the FP64 residual kernel:
    # both converge to the sequential solution, and to each other within the tolerance.
    kw = full(dict(CASES[case], tol=1e-11, init_guess=2))
    p = oprob(kw)
    u0 = synth.u0_uniform(p.nspace, -0.05, 0.05, 40 + case)
    res = {}
    for fx in (True, False):
        with pint.Solver(**kw) as s:
            s.set_fx_residual(fx)
            U = torch.zeros(p.nt, p.nspace, dtype=torch.float64, device="cuda")
            st = s.solve(dev(u0), U, check=False)
            assert st["rc"] == 0, st
            res[fx] = host(U)
    seq = O.sequential(p, u0)[-p.nt:]
    assert O.rel_err(res[True], seq) < 1e-9
    assert O.rel_err(res[True], res[False]) < 1e-9


def test_fx_residual_option_rejected_where_unsupported():
    # Eyre's splitting (its explicit Laplacian acts on u_{n-1}), cells that are not square
    # (no integer stencil) and FP64 handles keep the FP64 residual kernel
    for kw in (dict(equation="cahn_hilliard_eyre", dim=2, nx=16, ny=16, bc="neumann", eps=0.05, nt=8, T=8e-4),
               dict(equation="linear_ch", dim=2, nx=16, ny=8, bc="neumann", eps=0.05, beta=0.5, nt=8, T=1e-3)):
        with pint.Solver(**full(kw)) as s:
            with pytest.raises(pint.PintError):
                s.set_fx_residual(True)
    with pint.Solver(**full(dict(equation="cahn_hilliard", dim=2, nx=16, ny=16, bc="neumann", eps=0.05,
                                 nt=8, T=8e-4))) as s:
        s.set_fx_residual(True)   # the u^3 term is supported
    with pint.Solver(**full(dict(precision="fp64"))) as s:
        with pytest.raises(pint.PintError):
            s.set_fx_residual(True)
