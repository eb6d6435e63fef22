"""pint_residual_static: the residual entry point for callers that cannot
allocate device memory (its reduction scratch is a static device array).

Checked against pint_residual, the handle-based entry point, on two calls in a
row: the second call reuses the scratch the first one left behind.  This file
is collected last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

from paper_2304_14021_gb300 import build_lib, pint, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib.build()


CASES = [
    dict(equation="linear_ch", dim=2, nx=64, ny=48, bc="neumann", eps=0.05, beta=0.5, T=0.005, nt=16),
    dict(equation="cahn_hilliard", dim=2, nx=40, ny=40, bc="neumann", eps=0.05, T=8e-4, nt=8),
    dict(equation="biharmonic", dim=1, nx=64, ny=1, bc="ss", T=0.01, nt=32),
    # Crank-Nicolson and Eyre's splitting: the first level of ||b|| then comes from a one-level residual
    dict(equation="linear_ch", dim=2, nx=48, ny=32, bc="neumann", eps=0.05, beta=0.5, T=0.005, nt=8, theta=0.5),
    dict(equation="cahn_hilliard_eyre", dim=2, nx=32, ny=32, bc="neumann", eps=0.05, T=8e-4, nt=8),
    # the largest grid the library accepts (4096 x 1024 points): its residual grid is the largest
    dict(equation="linear_ch", dim=2, nx=4096, ny=1024, bc="neumann", eps=0.05, beta=0.5, T=1e-6, nt=2),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_static_residual_matches_handle_residual_twice(case):
    kw = dict(CASES[case], alpha=1e-2, tol=1e-8, max_iter=50, precision="fp64")
    ns = kw["nx"] * (kw["ny"] if kw["dim"] == 2 else 1)
    nt = kw["nt"]
    rel = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pint.Solver(**kw) as s:
        for call in range(2):                                  # two calls in a row
            u0 = torch.from_numpy(synth.u0_uniform(ns, -1, 1, 10 * case + call)).cuda()
            U = torch.from_numpy(synth.random_iterate(nt, ns, 20 * case + call)).cuda()
            r_ref = torch.empty(nt, ns, dtype=torch.float64, device="cuda")
            rel_ref = s.residual(u0, U, r_ref)
            r = torch.full((nt, ns), np.nan, dtype=torch.float64, device="cuda")
            rel.fill_(np.nan)
            pint.residual_static(u0, U, rel, r=r, **kw)
            torch.cuda.synchronize()
            scale = r_ref.abs().max().item()
            assert (r - r_ref).abs().max().item() <= 1e-13 * scale
            assert abs(rel.item() - rel_ref) <= 1e-12 * rel_ref


def test_static_residual_rejects_invalid_problem():
    rel = torch.zeros(1, dtype=torch.float64, device="cuda")
    u0 = torch.zeros(64, dtype=torch.float64, device="cuda")
    U = torch.zeros(32, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(pint.PintError) as e:
        pint.residual_static(u0, U, rel, equation="biharmonic", dim=1, nx=64, bc="ss", nt=48, T=0.01)
    assert e.value.code == pint.PINT_EINVAL
