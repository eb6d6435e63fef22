"""Pins for the CPU oracle: each test checks it against something other than
itself (closed forms, a library routine, brute force on tiny sizes, the
paper's convergence theory, the invariants of Cahn-Hilliard)."""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from oracle import pint_oracle as O
from paper_2304_14021_gb300 import synth


def P(**kw):
    return O.Problem(**kw)


# --- spatial spectra (Sec. 2.2.2 spectral discussion, Remark 2.5) -------------

@pytest.mark.parametrize("bc", ["ss", "neumann"])
@pytest.mark.parametrize("n", [5, 8, 13])
def test_laplacian_1d_spectrum_closed_form(bc, n):
    L = O.laplacian_1d(n, bc).toarray()
    h = 1.0 / (n + 1) if bc == "ss" else 1.0 / n
    if bc == "ss":
        lam = [-(4 / h**2) * np.sin(p * np.pi / (2 * (n + 1))) ** 2 for p in range(1, n + 1)]
    else:
        lam = [-(4 / h**2) * np.sin(p * np.pi / (2 * n)) ** 2 for p in range(n)]
    assert np.allclose(np.sort(np.linalg.eigvalsh(L)), np.sort(lam), rtol=1e-12, atol=1e-9)
    assert np.allclose(L, L.T)


@pytest.mark.parametrize("bc", ["ss", "neumann"])
def test_laplacian_2d_spectrum_and_modes(bc):
    p = P(dim=2, nx=6, ny=4, bc=bc)
    L = O.laplacian(p).toarray()
    # Eigenvectors are products of the 1-D sine / cosine modes.
    x, y = synth.grid_points_1d(6, bc), synth.grid_points_1d(4, bc)
    for (a, b) in [(1, 1), (2, 3), (4, 2)]:
        if bc == "ss":
            phi = np.outer(np.sin(b * np.pi * y), np.sin(a * np.pi * x)).ravel()
            lam = -(4 * 49) * np.sin(a * np.pi / 14) ** 2 - (4 * 25) * np.sin(b * np.pi / 10) ** 2
        else:
            a, b = a - 1, b - 1
            phi = np.outer(np.cos(b * np.pi * y), np.cos(a * np.pi * x)).ravel()
            lam = -(4 * 36) * np.sin(a * np.pi / 12) ** 2 - (4 * 16) * np.sin(b * np.pi / 8) ** 2
        assert np.allclose(L @ phi, lam * phi, atol=1e-9 * abs(lam) + 1e-10)


def test_neumann_laplacian_conserves_mass():
    # Column sums vanish: sum(Delta_h u) = 0 for any u (cell-centred Neumann).
    for p in [P(nx=9, bc="neumann"), P(dim=2, nx=5, ny=7, bc="neumann")]:
        L = O.laplacian(p)
        assert np.abs(np.asarray(L.sum(axis=0))).max() < 1e-9


# --- exact per-mode decay of the sequential scheme (Eq. 2.5, theta = 1) -------

@pytest.mark.parametrize("eq", [O.BIHARMONIC, O.LINEAR_CH])
@pytest.mark.parametrize("bc", ["ss", "neumann"])
def test_sequential_eigenmode_decay(eq, bc):
    n, nt, T, mode = 24, 12, 3e-4, 3
    p = P(equation=eq, nx=n, bc=bc, eps=0.05, beta=0.5, T=T, nt=nt)
    x = synth.grid_points_1d(n, bc)
    h = 1.0 / (n + 1) if bc == "ss" else 1.0 / n
    if bc == "ss":
        phi = np.sin(mode * np.pi * x)
        lam = -(4 / h**2) * np.sin(mode * np.pi / (2 * (n + 1))) ** 2
    else:
        phi = np.cos(mode * np.pi * x)
        lam = -(4 / h**2) * np.sin(mode * np.pi / (2 * n)) ** 2
    mu = lam**2 if eq == O.BIHARMONIC else 0.25 * lam + 0.0025 * lam**2
    U = O.sequential(p, phi)
    expect = np.array([(1 + p.dt * mu) ** (-(k + 1)) * phi for k in range(nt)])
    assert O.rel_err(U, expect) < 1e-12


def test_config1_closed_form():
    # 1-D biharmonic, simply supported, 64 vertices, u0 = sin(pi x) + 0.5 sin(3 pi x):
    # two exact sine modes, so U_n = sum_k a_k (1 + dt lambda_k^2)^{-n} sin(k pi x).
    n, nt, T = 64, 32, 0.01
    p = P(equation=O.BIHARMONIC, nx=n, bc="ss", T=T, nt=nt)
    u0 = synth.u0_sine_modes(n)
    U = O.sequential(p, u0)
    x = synth.grid_points_1d(n, "ss")
    h = 1.0 / 65
    ex = np.zeros_like(U)
    for k, a in [(1, 1.0), (3, 0.5)]:
        lam = -(4 / h**2) * np.sin(k * np.pi / 130) ** 2
        for m in range(nt):
            ex[m] += a * (1 + p.dt * lam**2) ** (-(m + 1)) * np.sin(k * np.pi * x)
    # cond(I + dt A) ~ 1e5 here, so each banded solve carries ~1e-11 roundoff.
    assert O.rel_err(U, ex) < 2e-11


def test_sequential_step_matches_library_sparse_solve():
    p = P(equation=O.LINEAR_CH, dim=2, nx=8, ny=8, bc="neumann", eps=0.05, beta=0.5, T=1e-3, nt=4)
    u0 = synth.u0_uniform(64, -0.05, 0.05, 3)
    U = O.sequential(p, u0)
    A = O.operator_A(p)
    M = (np.eye(64) / p.dt + A.toarray())
    u = u0.copy()
    for k in range(4):
        u = spla.spsolve(sps.csr_matrix(M), u / p.dt)
        assert np.allclose(U[k], u, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_sequential_at_selected_steps_matches_stepping(theta):
    # u_n = M^n u_0 by binary powering equals stepping the recurrence n times
    p = P(equation=O.LINEAR_CH, dim=2, nx=6, ny=5, bc="neumann", eps=0.05, beta=0.5, T=4e-3, nt=40, theta=theta)
    u0 = synth.u0_uniform(30, -0.05, 0.05, 5)
    U = O.sequential(p, u0)
    steps = [1, 2, 5, 17, 40]
    Us = O.sequential_linear_at(p, u0, steps)
    for i, n in enumerate(steps):
        assert O.rel_err(Us[i], U[n - 1]) < 1e-12


def test_sequential_at_long_axis_eigenmode_closed_form():
    # 1-D biharmonic, cell-centred Neumann, 64 cells, dt = 1e-6 over 2^20 steps:
    # a cosine mode decays by (1 + dt lambda^2)^{-n}, the constant mode stays put
    n, nt = 64, 1 << 20
    p = P(equation=O.BIHARMONIC, nx=n, bc="neumann", T=nt * 1e-6, nt=nt)
    x = synth.grid_points_1d(n, "neumann")
    h = 1.0 / n
    steps = [1, 1000, 1 << 19, 1 << 20]
    for mode in (1, 2):
        phi = np.cos(mode * np.pi * x)
        lam = -(4 / h**2) * np.sin(mode * np.pi / (2 * n)) ** 2
        Us = O.sequential_linear_at(p, 0.3 + phi, steps)
        for i, k in enumerate(steps):
            ex = 0.3 + (1 + p.dt * lam**2) ** (-k) * phi
            # M carries about cond(I + dt A) eps = 3e-14 of rounding, compounded over up
            # to 2^20 steps (1.2e-10 seen); a wrong power or step is off by O(1e-2) or more
            assert np.abs(Us[i] - ex).max() < 1e-9


# --- all-at-once system (Eq. 2.6-2.7) vs sequential --------------------------

@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("eq,bc,dim", [(O.BIHARMONIC, "ss", 1), (O.LINEAR_CH, "neumann", 1),
                                       (O.LINEAR_CH, "neumann", 2)])
def test_all_at_once_dense_equals_sequential(theta, eq, bc, dim):
    p = P(equation=eq, dim=dim, nx=6, ny=5, bc=bc, eps=0.1, beta=0.4, T=2e-3, nt=6, theta=theta)
    u0 = synth.u0_uniform(p.nspace, -1, 1, 7)
    assert O.rel_err(O.all_at_once_dense_linear(p, u0), O.sequential(p, u0)) < 1e-11


def test_ch_newton_step_at_rounding_floor_solves_the_step():
    # eps = 0.1, 128 cells, dt = 1e-4 (cond(J) ~ 4e3): the 1e-14 update test is out of
    # reach, the rounding-floor stop ends Newton; the step equation then holds to rounding
    p = P(equation=O.CAHN_HILLIARD, nx=128, bc="neumann", eps=0.1, T=1e-4, nt=1)
    x = synth.grid_points_1d(128, "neumann")
    u0 = 0.75 * np.sin(2 * np.pi * x) + 0.25 * np.cos(4 * np.pi * x)
    u, it = O.ch_step_newton(p, u0)
    L = O.laplacian(p)
    F = (u - u0) / p.dt - L @ (u ** 3 - u) + p.eps ** 2 * (L @ (L @ u))
    scale = np.abs(u0 / p.dt).max() + np.abs(p.eps ** 2 * (L @ (L @ u))).max()
    assert it <= 10 and np.abs(F).max() < 1e-12 * scale


def test_ch_all_at_once_newton_equals_sequential():
    p = P(equation=O.CAHN_HILLIARD, nx=12, bc="neumann", eps=0.1, T=4e-3, nt=5)
    u0 = 0.6 * np.cos(np.pi * synth.grid_points_1d(12, "neumann")) + 0.1
    assert O.rel_err(O.all_at_once_newton_ch(p, u0), O.sequential(p, u0)) < 1e-11


@pytest.mark.parametrize("eq", [O.BIHARMONIC, O.LINEAR_CH, O.CAHN_HILLIARD])
def test_residual_vanishes_at_sequential_and_equals_b_at_zero(eq):
    bc = "ss" if eq == O.BIHARMONIC else "neumann"
    p = P(equation=eq, dim=2, nx=6, ny=6, bc=bc, eps=0.1, beta=0.5, T=2e-3, nt=4)
    u0 = synth.u0_ch(36, 1, amp=0.5)
    U = O.sequential(p, u0)
    r = O.residual(p, u0, U)
    scale = np.abs(U).max() / p.dt
    assert np.abs(r).max() < 1e-11 * scale
    r0 = O.residual(p, u0, np.zeros_like(U))
    assert np.allclose(r0[0], u0 / p.dt) and np.all(r0[1:] == 0)
    assert np.isclose(O.rhs_norm(p, u0), np.linalg.norm(u0) / p.dt)


# --- the iteration: paper form (Eq. 2.6) vs residual form ---------------------

@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_paper_form_iterates_equal_residual_form(theta):
    p = P(equation=O.LINEAR_CH, nx=7, bc="neumann", eps=0.08, beta=0.5, T=5e-3, nt=6,
          theta=theta, alpha=0.05)
    u0 = synth.u0_uniform(7, -1, 1, 2)
    U0 = synth.random_iterate(6, 7, 4)
    a = O.pint_iteration_paper_form(p, u0, U0, 5)
    b = O.pint_iteration_residual_form(p, u0, U0, 5)
    for x, y in zip(a, b):
        assert O.rel_err(x, y) < 1e-12


@pytest.mark.parametrize("eq,dim,theta", [(O.BIHARMONIC, 1, 1.0), (O.LINEAR_CH, 2, 1.0),
                                          (O.LINEAR_CH, 1, 0.5), (O.CAHN_HILLIARD, 2, 1.0)])
def test_diagonalized_steps_equal_dense_preconditioner(eq, dim, theta):
    # Steps 1-3 of Eq. 2.8 (Eq. 4.14) with the Lemma 2.1 eigenvalues == dense P_alpha^{-1}.
    bc = "ss" if eq == O.BIHARMONIC else "neumann"
    p = P(equation=eq, dim=dim, nx=6, ny=4, bc=bc, eps=0.1, beta=0.5, T=3e-3, nt=8,
          theta=theta, alpha=0.02)
    r = synth.random_iterate(8, p.nspace, 11)
    jb = 0.7 if eq == O.CAHN_HILLIARD else None
    d1 = O.diagonalized_apply(p, p.alpha, r, jb)
    d2 = O.precond_dense(p, p.alpha, r, jb)
    assert O.rel_err(d1, d2) < 1e-11


def test_preconditioner_is_exact_solver_at_alpha_zero_limit():
    # P_alpha -> K as alpha -> 0: one iteration from U = 0 with tiny alpha lands
    # on the sequential solution up to O(alpha).
    p = P(equation=O.BIHARMONIC, nx=10, bc="ss", T=1e-3, nt=8, alpha=1e-9)
    u0 = synth.u0_sine_modes(10)
    U1 = O.pint_iteration_residual_form(p, u0, np.zeros((8, 10)), 1)[0]
    assert O.rel_err(U1, O.sequential(p, u0)) < 1e-7


# --- convergence theory (Eq. 2.17-2.18, Thm 2.4, Thm 3.3) ----------------------

def _signed_mode_factors(p):
    """-alpha R^N / (1 - alpha R^N) per eigenmode of A (Eq. 2.18), R = 1/(1 + dt mu)."""
    mu, Q = np.linalg.eigh(O.operator_A(p).toarray())
    RN = (1.0 / (1.0 + p.dt * mu)) ** p.nt
    return -p.alpha * RN / (1.0 - p.alpha * RN), Q


@pytest.mark.parametrize("eq,bc,alpha", [(O.BIHARMONIC, "ss", 0.05), (O.BIHARMONIC, "neumann", 0.05),
                                         (O.LINEAR_CH, "neumann", 0.05), (O.LINEAR_CH, "neumann", 0.2)])
def test_per_mode_error_recurrence_and_bounds(eq, bc, alpha):
    # From the second iterate on, each spatial eigenmode of the last-level error
    # is multiplied by exactly -alpha R^N/(1 - alpha R^N) per iteration (Eq. 2.17-2.18).
    p = P(equation=eq, nx=8, bc=bc, eps=0.08, beta=0.5, T=0.02, nt=8, alpha=alpha)
    u0 = synth.u0_uniform(8, -1, 1, 9)
    Useq = O.sequential(p, u0)
    its = O.pint_iteration_paper_form(p, u0, synth.random_iterate(8, 8, 5), 5)
    fac, Q = _signed_mode_factors(p)
    E = [Q.T @ (U[-1] - Useq[-1]) for U in its]
    checked = 0
    for k in range(1, 4):
        # roundoff in U (~1e-15) bounds how well a small mode's ratio is resolved
        floor = 1e-12 * np.abs(E[0]).max()
        assert np.all(np.abs(E[k] - fac * E[k - 1]) <= 1e-6 * np.abs(E[k - 1]) + floor)
        checked += int((np.abs(E[k]) > 1e3 * floor).sum())
    assert checked >= 3
    exact = O.mode_contraction(p)
    assert np.isclose(exact, np.abs(fac).max(), rtol=1e-12)
    if eq == O.BIHARMONIC:
        assert exact <= O.thm_bound_biharmonic(alpha) * (1 + 1e-12)
        if bc == "neumann":     # constant mode: mu = 0, R = 1, factor alpha/(1-alpha)
            assert np.isclose(exact, alpha / (1 - alpha), rtol=1e-12)
    else:
        assert exact <= O.thm_bound_linear_ch(p) * (1 + 1e-9)


def test_config2_contraction_close_to_thm33_bound():
    # 2-D linearized CH, 256^2 cell-centred Neumann, beta=0.5, eps=0.05, N_t=128, T=0.1.
    for alpha in (1e-2, 1e-3):
        p = P(equation=O.LINEAR_CH, dim=2, nx=256, ny=256, bc="neumann", eps=0.05, beta=0.5,
              T=0.1, nt=128, alpha=alpha)
        exact, bound = O.mode_contraction(p), O.thm_bound_linear_ch(p)
        assert exact <= bound
        assert exact > 0.999 * bound      # the discrete spectrum nearly hits z*
        assert 0.9 * alpha < exact < 2.5 * alpha


# --- Cahn-Hilliard invariants (Eq. 1.5) ---------------------------------------

def test_ch_mass_conserved_energy_decreasing_2d():
    p = P(equation=O.CAHN_HILLIARD, dim=2, nx=16, ny=16, bc="neumann", eps=0.05, T=2.4e-3, nt=24)
    u0 = synth.u0_ch(256, 0)
    U = O.sequential(p, u0)
    m0 = O.discrete_mass(p, u0)
    assert max(abs(O.discrete_mass(p, u) - m0) for u in U) < 1e-12
    E = [O.discrete_energy(p, u0)] + [O.discrete_energy(p, u) for u in U]
    assert all(E[i + 1] <= E[i] + 1e-14 for i in range(len(E) - 1))
    assert E[-1] < E[0]


@pytest.mark.parametrize("case", ["1d", "2d_x", "2d_y"])
def test_discrete_energy_closed_form_cosine_mode(case):
    # One cosine mode a cos(p pi x) on the cell-centred grid (h = 1/n, x_i = (i + 1/2) h) with 0 < 4p < 2n:
    # sum_i cos^2 = n/2, sum_i cos^4 = 3n/8, and the face differences are
    # -2a sin(p pi h/2) sin(p pi j/n), j = 1..n-1, whose squares sum to 2 n a^2 sin^2(p pi/(2n)).
    # So the bulk part is (3a^4/8 - a^2 + 1)/4 and the gradient part eps^2 n^2 a^2 sin^2(p pi/(2n)),
    # in 1-D and 2-D alike (a mode constant along the other axis), which fixes the weight between the
    # two sums, the power of h, and the face sums of each axis.
    n, pm, a, eps = 16, 3, 0.7, 0.05
    x = (np.arange(n) + 0.5) / n
    mode = a * np.cos(pm * np.pi * x)
    if case == "1d":
        p, u = P(equation=O.CAHN_HILLIARD, dim=1, nx=n, bc="neumann", eps=eps), mode
    elif case == "2d_x":
        p, u = P(equation=O.CAHN_HILLIARD, dim=2, nx=n, ny=n, bc="neumann", eps=eps), np.tile(mode, n)
    else:
        p, u = P(equation=O.CAHN_HILLIARD, dim=2, nx=n, ny=n, bc="neumann", eps=eps), np.repeat(mode, n)
    bulk = (3 * a**4 / 8 - a**2 + 1) / 4
    grad = eps**2 * n**2 * a**2 * np.sin(pm * np.pi / (2 * n)) ** 2
    assert abs(O.discrete_energy(p, u) - (bulk + grad)) < 1e-14
    # the constant states +-1 have zero energy; the constant 0 has h^d sum 1/4 = 1/4
    assert abs(O.discrete_energy(p, np.ones(p.nspace))) < 1e-15
    assert abs(O.discrete_energy(p, np.zeros(p.nspace)) - 0.25) < 1e-15


def test_thm33_bound_rejects_negative_beta():
    # Theorem 3.3's maximizer z* = beta^2 dt/(2 eps^2) belongs to the anti-diffusive term (beta >= 0)
    with pytest.raises(ValueError):
        O.thm_bound_linear_ch(P(equation=O.LINEAR_CH, dim=1, nx=16, bc="neumann", beta=-0.5, eps=0.05,
                                T=0.1, nt=16))


def test_ch_constant_state_is_stationary():
    p = P(equation=O.CAHN_HILLIARD, dim=2, nx=8, ny=8, bc="neumann", eps=0.02, T=1e-3, nt=5)
    u0 = np.full(64, 0.3)
    assert np.abs(O.sequential(p, u0) - 0.3).max() < 1e-14


def test_ch_newton_step_solves_the_be_equation():
    p = P(equation=O.CAHN_HILLIARD, nx=32, bc="neumann", eps=0.05, T=1e-4, nt=1)
    u0 = synth.u0_ch(32, 4, amp=0.8)
    u1, its = O.ch_step_newton(p, u0)
    L = O.laplacian(p).toarray()
    F = (u1 - u0) / p.dt - L @ (u1**3 - u1) + p.eps**2 * L @ L @ u1
    assert np.abs(F).max() < 1e-9 * np.abs(u0).max() / p.dt
    assert its <= 10


def test_ch_iteration_converges_to_sequential():
    # PinT-I (one quasi-Newton step per WR step, scalar averaged Jacobian)
    # reaches the sequential BE solution (the fixed point is unchanged).
    p = P(equation=O.CAHN_HILLIARD, nx=16, bc="neumann", eps=0.1, T=4e-3, nt=8, alpha=0.01)
    u0 = 0.5 * np.cos(np.pi * synth.grid_points_1d(16, "neumann"))
    Useq = O.sequential(p, u0)
    its = O.pint_iteration_residual_form(p, u0, np.tile(u0, (8, 1)), 40, dense=False)
    assert O.rel_err(its[-1], Useq) < 1e-11


@pytest.mark.parametrize("kw", [
    dict(equation="linear_ch", dim=2, nx=12, ny=8, bc="neumann", eps=0.05, beta=0.5, T=0.01, nt=8),
    dict(equation="biharmonic", dim=2, nx=7, ny=9, bc="ss", T=1e-3, nt=4),
    dict(equation="cahn_hilliard", dim=2, nx=8, ny=8, bc="neumann", eps=0.05, T=8e-4, nt=8),
    dict(equation="linear_ch", dim=1, nx=20, bc="neumann", eps=0.05, beta=0.5, T=0.01, nt=16),
])
def test_separable_apply_matches_dense_eigendecomposition(kw):
    # The tensor-product eigenbasis (1-D eigh of Delta_x, Delta_y) and the dense
    # eigh of the 2-D operator give the same P_alpha^{-1} r (Remark 2.5).
    p = O.Problem(**kw)
    r = synth.random_iterate(p.nt, p.nspace, 5)
    a = O.diagonalized_apply(p, 1e-2, r, 0.4)
    b = O.diagonalized_apply_separable(p, 1e-2, r, 0.4)
    assert O.rel_err(b, a) < 1e-12


# --- vertex-centred Neumann (the paper's Delta_h, Eq. 2.4) --------------------

@pytest.mark.parametrize("n", [5, 8, 13])
def test_vertex_neumann_laplacian_spectrum_and_modes(n):
    # End rows (-2, 2)/h^2 on n vertices, h = 1/(n-1): not symmetric, but similar
    # to a symmetric matrix through W = diag(1/2, 1, ..., 1, 1/2); eigenpairs
    # cos(p pi x_j), -(4/h^2) sin^2(p pi / (2(n-1))).
    L = O.laplacian_1d(n, "neumann_v").toarray()
    h = 1.0 / (n - 1)
    assert L[0, 1] == 2.0 / h**2 and L[-1, -2] == 2.0 / h**2 and L[0, 0] == -2.0 / h**2
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    S = np.diag(np.sqrt(w)) @ L @ np.diag(1.0 / np.sqrt(w))
    assert np.allclose(S, S.T, atol=1e-9)
    x = synth.grid_points_1d(n, "neumann_v")
    assert x[0] == 0.0 and x[-1] == 1.0
    for p in range(n):
        phi = np.cos(p * np.pi * x)
        lam = -(4 / h**2) * np.sin(p * np.pi / (2 * (n - 1))) ** 2
        assert np.allclose(L @ phi, lam * phi, atol=1e-9 * (abs(lam) + 1))
    assert np.allclose(np.sort(O.laplacian_eigs_1d(n, "neumann_v")), np.sort(np.linalg.eigvals(L).real),
                       rtol=1e-10, atol=1e-8)


@pytest.mark.parametrize("eq", [O.BIHARMONIC, O.LINEAR_CH])
@pytest.mark.parametrize("dim", [1, 2])
def test_vertex_neumann_eigenmode_decay(eq, dim):
    n, nt, T = 13, 10, 3e-4
    p = P(equation=eq, dim=dim, nx=n, ny=9, bc="neumann_v", eps=0.05, beta=0.5, T=T, nt=nt)
    x, y = synth.grid_points_1d(n, "neumann_v"), synth.grid_points_1d(9, "neumann_v")
    a, b = 3, 2
    lam = -(4 * (n - 1) ** 2) * np.sin(a * np.pi / (2 * (n - 1))) ** 2
    phi = np.cos(a * np.pi * x)
    if dim == 2:
        lam += -(4 * 8**2) * np.sin(b * np.pi / 16) ** 2
        phi = np.outer(np.cos(b * np.pi * y), np.cos(a * np.pi * x)).ravel()
    mu = lam**2 if eq == O.BIHARMONIC else 0.25 * lam + 0.0025 * lam**2
    U = O.sequential(p, phi)
    expect = np.array([(1 + p.dt * mu) ** (-(k + 1)) * phi for k in range(nt)])
    assert O.rel_err(U, expect) < 1e-11


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("dim", [1, 2])
def test_vertex_neumann_all_at_once_and_diagonalized(theta, dim):
    p = P(equation=O.LINEAR_CH, dim=dim, nx=7, ny=5, bc="neumann_v", eps=0.1, beta=0.4, T=2e-3, nt=6,
          theta=theta, alpha=0.02)
    u0 = synth.u0_uniform(p.nspace, -1, 1, 7)
    assert O.rel_err(O.all_at_once_dense_linear(p, u0), O.sequential(p, u0)) < 1e-11
    r = synth.random_iterate(6, p.nspace, 11)
    d_dense = O.precond_dense(p, p.alpha, r)
    assert O.rel_err(O.diagonalized_apply(p, p.alpha, r), d_dense) < 1e-10
    assert O.rel_err(O.diagonalized_apply_separable(p, p.alpha, r), d_dense) < 1e-10


def test_vertex_neumann_ch_diagonalized_and_constant_state():
    p = P(equation=O.CAHN_HILLIARD, dim=2, nx=6, ny=5, bc="neumann_v", eps=0.1, T=3e-3, nt=8, alpha=0.02)
    r = synth.random_iterate(8, p.nspace, 12)
    assert O.rel_err(O.diagonalized_apply(p, p.alpha, r, 0.7), O.precond_dense(p, p.alpha, r, 0.7)) < 1e-10
    u0 = np.full(p.nspace, 0.3)
    U = O.sequential(p, u0)
    assert np.abs(U - 0.3).max() < 1e-12


@pytest.mark.parametrize("bc", ["ss", "neumann", "neumann_v"])
def test_signed_beta_squared_eigenmode_decay(bc):
    # beta < 0 carries a negative beta^2: A = -0.25 Lap + eps^2 Lap^2, every mode decays
    # with (1 + dt mu)^(-n), mu = -0.25 lam + 0.0025 lam^2 > 0.
    n, nt, T, mode = 24, 12, 3e-3, 3
    p = P(equation=O.LINEAR_CH, nx=n, bc=bc, eps=0.05, beta=-0.5, T=T, nt=nt)
    x = synth.grid_points_1d(n, bc)
    h = O.grid_h(n, bc)
    if bc == "ss":
        phi = np.sin(mode * np.pi * x)
        lam = -(4 / h**2) * np.sin(mode * np.pi / (2 * (n + 1))) ** 2
    elif bc == "neumann":
        phi = np.cos(mode * np.pi * x)
        lam = -(4 / h**2) * np.sin(mode * np.pi / (2 * n)) ** 2
    else:
        phi = np.cos(mode * np.pi * x)
        lam = -(4 / h**2) * np.sin(mode * np.pi / (2 * (n - 1))) ** 2
    mu = -0.25 * lam + 0.0025 * lam**2
    assert mu > 0
    U = O.sequential(p, phi)
    expect = np.array([(1 + p.dt * mu) ** (-(k + 1)) * phi for k in range(nt)])
    assert O.rel_err(U, expect) < 1e-11
    r = synth.random_iterate(nt, n, 3)
    assert O.rel_err(O.diagonalized_apply(p, 0.02, r), O.precond_dense(p, 0.02, r)) < 1e-10


# --- Cahn-Hilliard with Eyre's splitting (PinT-II, Sec. 4.2) -------------------

def _eyre(**kw):
    d = dict(equation=O.CAHN_HILLIARD_EYRE, dim=1, nx=12, bc="neumann", eps=0.1, T=4e-3, nt=5)
    d.update(kw)
    return P(**d)


def test_eyre_all_at_once_newton_equals_sequential_and_residual_vanishes():
    p = _eyre()
    u0 = 0.6 * np.cos(np.pi * synth.grid_points_1d(12, "neumann")) + 0.1
    Useq = O.sequential(p, u0)
    assert O.rel_err(O.all_at_once_newton_eyre(p, u0), Useq) < 1e-11
    assert np.abs(O.residual(p, u0, Useq)).max() < 1e-9 * np.abs(u0).max() / p.dt
    # at U = 0 the residual is b: b_1 = u0/dt - Delta u0, zero below
    R0 = O.residual(p, u0, np.zeros((p.nt, p.nspace)))
    L = O.laplacian(p)
    assert np.allclose(R0[0], u0 / p.dt - L @ u0, rtol=1e-13, atol=1e-9)
    assert np.abs(R0[1:]).max() == 0.0


def test_eyre_step_is_the_split_scheme():
    # one step solves (u - u_prev)/dt = Delta(u^3) - Delta u_prev - eps^2 Delta^2 u (convex part
    # implicit, concave part explicit), written out with dense matrices
    p = _eyre(nx=9, nt=1, T=1e-3)
    u_prev = synth.u0_uniform(9, -0.8, 0.8, 5)
    u = O.sequential(p, u_prev)[0]
    L = O.laplacian(p).toarray()
    lhs = (u - u_prev) / p.dt
    rhs = L @ u ** 3 - L @ u_prev - p.eps ** 2 * L @ (L @ u)
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-8)


def test_eyre_unconditionally_energy_stable_and_mass_conserving():
    # Eyre's scheme decreases the discrete energy for any dt (here dt = 1e-2 >> eps^2 = 1e-3)
    p = _eyre(dim=2, nx=10, ny=10, eps=0.0316, T=0.2, nt=20)
    u0 = synth.u0_ch(100, 3)
    U = O.sequential(p, u0)
    E = [O.discrete_energy(p, u0)] + [O.discrete_energy(p, u) for u in U]
    assert all(E[i + 1] <= E[i] + 1e-12 for i in range(len(E) - 1))
    m0 = O.discrete_mass(p, u0)
    assert max(abs(O.discrete_mass(p, u) - m0) for u in U) < 1e-12


def test_eyre_diagonalized_equals_dense_and_iteration_converges():
    p = _eyre(dim=2, nx=6, ny=5, nt=8, T=3e-3, alpha=0.02)
    r = synth.random_iterate(8, p.nspace, 13)
    d_dense = O.precond_dense(p, p.alpha, r, 0.6)
    assert O.rel_err(O.diagonalized_apply(p, p.alpha, r, 0.6), d_dense) < 1e-10
    assert O.rel_err(O.diagonalized_apply_separable(p, p.alpha, r, 0.6), d_dense) < 1e-10
    u0 = synth.u0_ch(p.nspace, 4)
    its = O.pint_iteration_residual_form(p, u0, np.tile(u0, (p.nt, 1)), 12)
    assert O.rel_err(its[-1], O.sequential(p, u0)) < 1e-10


def test_eyre_constant_state_is_stationary():
    p = _eyre(dim=2, nx=6, ny=6)
    U = O.sequential(p, np.full(36, -0.4))
    assert np.abs(U + 0.4).max() < 1e-13


# --- space-varying averaged Jacobian (Eq. 4.12, paper-literal PinT-I/II) -------

@pytest.mark.parametrize("eq", [O.CAHN_HILLIARD, O.CAHN_HILLIARD_EYRE])
def test_varying_jacobian_apply_equals_dense_and_reduces_to_scalar(eq):
    p = P(equation=eq, dim=2, nx=6, ny=5, bc="neumann", eps=0.1, T=3e-3, nt=8, alpha=0.02)
    r = synth.random_iterate(8, p.nspace, 21)
    jt = synth.u0_uniform(p.nspace, 0.0, 3.0, 22)
    d = O.diagonalized_apply_varying(p, p.alpha, r, jt)
    assert O.rel_err(d, np.linalg.solve(O.dense_P_varying(p, p.alpha, jt), r.ravel()).reshape(r.shape)) < 1e-10
    const = np.full(p.nspace, 0.7)
    assert O.rel_err(O.diagonalized_apply_varying(p, p.alpha, r, const),
                     O.precond_dense(p, p.alpha, r, 0.7)) < 1e-10


def test_varying_jacobian_iteration_converges_faster_on_separated_phases():
    # phase-separated data (|u| near 1 away from an interface): the space-varying J~
    # tracks the Jacobian where the scalar mean cannot, so the iteration contracts faster
    p = P(equation=O.CAHN_HILLIARD, dim=1, nx=48, bc="neumann", eps=0.04, T=8e-3, nt=16, alpha=0.01)
    x = synth.grid_points_1d(48, "neumann")
    u0 = np.tanh((x - 0.5) / (np.sqrt(2) * 0.04)) + 0.05 * np.cos(3 * np.pi * x)
    ref = O.sequential(p, u0)
    U0 = np.tile(u0, (p.nt, 1))
    ev = [O.rel_err(U, ref) for U in O.pint_iteration_varying(p, u0, U0, 6)]
    es = [O.rel_err(U, ref) for U in O.pint_iteration_residual_form(p, u0, U0, 6, dense=False)]
    assert ev[-1] < 1e-8
    assert ev[3] < es[3]


# --- the iteration counts the paper states (tests/golden/paper_iteration_counts.json) ---

def _paper_counts():
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_iteration_counts.json")) as f:
        return json.load(f)


def test_paper_four_iterations_at_a_million_steps_follow_from_the_contraction():
    # Neumann biharmonic: the constant mode contracts by alpha/(1-alpha) per iteration
    # (Eq. 2.18 with R = 1), so an O(1) initial error needs exactly the paper's count to
    # fall below its tolerance (and one fewer does not)
    gold = _paper_counts()["biharmonic_1d_dt1e-6"]
    nt = 1 << 20
    p = P(equation=O.BIHARMONIC, nx=64, bc="neumann", T=nt * 1e-6, nt=nt, alpha=1e-3)
    q = O.mode_contraction(p)
    assert abs(q - 1e-3 / (1 - 1e-3)) < 1e-12
    k = gold["iterations"]
    assert q ** k < gold["tolerance"] <= q ** (k - 1)


def test_paper_pint1_example_essentially_converged_after_four_iterations():
    # the oracle's PinT-I iteration with the space-varying Jacobian (Eq. 4.12), exact inner
    # solves, from a random iterate, at the paper's h, eps, dt and alpha (over 256 steps here
    # to keep the CPU suite short; the GPU test runs 1024): within 5e-3 of the sequential
    # solution in L^inf(0,T; L^2) after the paper's four iterations, and closer with the
    # varying Jacobian than with its scalar mean
    its = _paper_counts()["pint1_cahn_hilliard_1d"]["iterations"]
    nt, n = 256, 128
    p = P(equation=O.CAHN_HILLIARD, nx=n, bc="neumann", eps=0.1, T=nt * 1e-4, nt=nt, alpha=0.005)
    x = synth.grid_points_1d(n, "neumann")
    u0 = 0.75 * np.sin(2 * np.pi * x) + 0.25 * np.cos(4 * np.pi * x)
    seq = O.sequential(p, u0)
    Ui = synth.random_iterate(nt, n, 5)

    def err(U):
        return np.sqrt(np.sum((U - seq) ** 2, axis=1) / n).max()

    ev = err(O.pint_iteration_varying(p, u0, Ui, its)[-1])
    es = err(O.pint_iteration_residual_form(p, u0, Ui, its, dense=False)[-1])
    assert ev < 5e-3 and ev < es, (ev, es)


def test_golden_config3_64_fixture_is_consistent():
    # The stored oracle values of the 64 x 64 Cahn-Hilliard schedule (written by
    # tests/golden/make_ch_config3_64.py from oracle/ only) keep the invariants the oracle is pinned
    # to: zero mass (u0 has zero mean), energy decreasing from level to level and below E(u0).
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ch_config3_64x64.json")
    with open(path) as f:
        g = json.load(f)
    c = g["case"]
    p = P(equation=O.CAHN_HILLIARD, dim=2, nx=c["nx"], ny=c["ny"], bc="neumann", eps=c["eps"],
          T=c["nt"] * c["n_windows"] * c["dt"], nt=c["nt"], n_windows=c["n_windows"])
    u0 = synth.u0_ch(p.nspace, 0)
    assert max(abs(m) for m in g["mass"]) < 1e-12
    E = g["energy"]
    assert all(E[i + 1] <= E[i] for i in range(len(E) - 1)) and E[0] < O.discrete_energy(p, u0)
    assert len(g["window_ends"]) == c["n_windows"] and all(len(w["values"]) == p.nspace // g["sample_every_point"]
                                                            for w in g["window_ends"])
    # the first stored level is reproduced by the oracle's own step (a cheap end-to-end check of the file)
    u = u0.copy()
    for _ in range(g["levels"][0]):
        u, _ = O.ch_step_newton(p, u)
    assert abs(O.discrete_energy(p, u) - E[0]) < 1e-13 * E[0]
