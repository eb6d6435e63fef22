"""CPU oracle for the diagonalization-based parallel-in-time (PinT) method of
Garai & Mandal, "Diagonalization Based Parallel-in-Time Method for a Class of
Fourth Order Time Dependent PDEs" (arXiv 2304.14021).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path (no kernels, tables, helpers or constants); both sides receive the
same plain problem parameters and the same seeded input arrays.

Everything here is plain FP64 numpy/scipy.  Library primitives used as steps:
``scipy.linalg.lapack.dgbtrf/dgbtrs`` (banded LU), ``numpy.linalg.solve``
(dense LU), ``numpy.linalg.eigh`` and ``numpy.fft`` (only in the
``diagonalized_*`` functions, which restate the paper's three steps).

What is computed (section / equation numbers of the paper):

* Spatial operators: the centred finite-difference Laplacian Delta_h
  (Sec. 2.1, Eq. 2.4) for two boundary treatments,
  - ``bc="ss"``: simply supported u = Laplace(u) = 0 (the paper's boundary
    condition (ii) in Sec. 5.1), vertex grid of n interior points,
    h = 1/(n+1), zero ghost values for u and for Delta_h u;
  - ``bc="neumann"``: homogeneous Neumann d_nu u = d_nu Laplace(u) = 0 on a
    cell-centred grid of n cells, h = 1/n, mirror ghost values;
  - ``bc="neumann_v"``: the same conditions on the paper's own vertex grid
    (Eq. 2.4): n points x_j = j h including both ends, h = 1/(n-1), ghosts
    u_{-1} = u_1 and u_n = u_{n-2}, so the end rows read (-2, 2)/h^2.
  2-D operators are Kronecker sums (Remark 2.5).
* A = Delta_h^2 (biharmonic, Eq. 2.3), A = beta^2 Delta_h + eps^2 Delta_h^2 (beta^2 is
  signed: the field beta carries its sign, beta^2 := beta |beta|, so beta < 0 gives the
  diffusive second-order term of the general fourth-order problem of Sec. 3)
  (linearized Cahn-Hilliard, Sec. 3, Eq. 3.1).
* The sequential theta-method solution (Eq. 2.5 with alpha = 0): this is the
  fixed point the PinT iteration converges to (Sec. 2, after Eq. 2.2; the
  stopping rule of Sec. 5 measures the error against it).
* Nonlinear Cahn-Hilliard, fully implicit backward Euler (Eq. 4.5) solved per
  step by Newton's method with the exact Jacobian (Eq. 4.10 restricted to one
  time step, with J_s = diag(3 u^2)).
* The all-at-once residual b - K U (Eq. 2.6 / Eq. 4.8 with alpha = 0).
* Dense constructions on tiny sizes: the all-at-once matrix (Eq. 2.6-2.7), the
  alpha-circulant preconditioner P_alpha and the paper's literal WR iteration
  P_alpha U^k = b^{k-1}.
* The paper's three diagonalized steps (Eq. 2.8 / Eq. 4.14) with numpy's FFT,
  for long time axes where dense P_alpha is infeasible.
* Per-mode contraction factor of the fully discrete iteration (Eq. 2.17-2.18,
  Thm 2.4; Thm 3.3 for its linearized-CH bound), discrete energy and mass
  (Eq. 1.5).

Readings of the paper taken here:

* The diagonal of D_1 (Lemma 2.1) is computed from the DFT convention used in
  Step 1: with forward transform exp(-2 pi i n k / N_t) it is
  lambda_{1,k} = (1 - alpha^{1/N_t} exp(-2 pi i k/N_t)) / dt; the printed
  lambda_{1,n} omits the 1/dt of C_1.
* b^{k-1} (after Eq. 2.7) is read as (I/dt - (1-theta) A)(u_0 - alpha u_{N_t}^{k-1})
  in the first block.
* J_s(u) = diag(3 u^2) (the derivative of u^3 in Eq. 4.7; the printed
  "(3u)^2" is read as 3u^2).
* For the PinT-I preconditioner the averaged Jacobian J~ (Eq. 4.12) is taken
  as the scalar mean of 3u^2 over all space-time points ("jbar").  The fixed
  point is unchanged because the residual uses the exact nonlinearity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.linalg import lapack

BIHARMONIC = "biharmonic"
LINEAR_CH = "linear_ch"
CAHN_HILLIARD = "cahn_hilliard"
# Cahn-Hilliard with Eyre's convex-concave splitting (PinT-II, Sec. 4.2): u^3
# implicit, the concave -u part explicit.
CAHN_HILLIARD_EYRE = "cahn_hilliard_eyre"
CH_EQUATIONS = (CAHN_HILLIARD, CAHN_HILLIARD_EYRE)


@dataclass
class Problem:
    """Problem statement: the fields of Eq. 2.1 / 3.1 / 4.1 plus the
    discretization of Sec. 2.1 and the PinT parameter alpha (Eq. 2.2)."""
    equation: str = BIHARMONIC
    dim: int = 1
    nx: int = 16
    ny: int = 1
    bc: str = "ss"              # "ss" (simply supported), "neumann" (cell-centred) or "neumann_v" (vertex)
    eps: float = 1.0
    beta: float = 0.0
    T: float = 0.01
    nt: int = 8                 # time steps per window
    n_windows: int = 1
    theta: float = 1.0
    alpha: float = 1e-2
    extra: dict = field(default_factory=dict)

    @property
    def dt(self) -> float:
        return self.T / (self.nt * self.n_windows)

    @property
    def nspace(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)


# ----------------------------------------------------------------------------
# Spatial operators (Sec. 2.1, Eq. 2.4; Remark 2.5 for 2-D)
# ----------------------------------------------------------------------------

def grid_h(n: int, bc: str) -> float:
    """Mesh width on [0, 1]: vertex grid (n interior points) for "ss",
    cell-centred grid (n cells) for "neumann"."""
    if bc == "ss":
        return 1.0 / (n + 1)
    if bc == "neumann":
        return 1.0 / n
    if bc == "neumann_v":
        return 1.0 / (n - 1)
    raise ValueError(bc)


def grid_points(n: int, bc: str) -> np.ndarray:
    h = grid_h(n, bc)
    if bc == "ss":
        return h * np.arange(1, n + 1)
    if bc == "neumann_v":
        return h * np.arange(n)
    return h * (np.arange(n) + 0.5)


def laplacian_1d(n: int, bc: str) -> sp.csr_matrix:
    """Centred second difference (u_{j-1} - 2u_j + u_{j+1}) / h^2 (Eq. 2.4).

    "ss": ghosts u_0 = u_{n+1} = 0.  "neumann" (cell-centred): mirror ghosts
    u_{-1} = u_0, u_n = u_{n-1}, so the end rows read (-1, 1)/h^2.
    """
    h = grid_h(n, bc)
    main = -2.0 * np.ones(n)
    if bc == "neumann":
        main[0] = -1.0
        main[-1] = -1.0
    up = np.ones(n - 1)
    lo = np.ones(n - 1)
    if bc == "neumann_v":   # u_{-1} = u_1, u_n = u_{n-2}: end rows (-2, 2), not symmetric
        up[0] = 2.0
        lo[-1] = 2.0
    return sp.diags([lo, main, up], [-1, 0, 1], format="csr") / (h * h)


def laplacian(p: Problem) -> sp.csr_matrix:
    """Delta_h on the 1-D or 2-D grid; index = y * nx + x (x fastest).
    2-D: I (x) Delta_x + Delta_y (x) I (Remark 2.5)."""
    lx = laplacian_1d(p.nx, p.bc)
    if p.dim == 1:
        return lx
    ly = laplacian_1d(p.ny, p.bc)
    return (sp.kron(sp.identity(p.ny), lx) + sp.kron(ly, sp.identity(p.nx))).tocsr()


def operator_A(p: Problem) -> sp.csr_matrix:
    """Linear spatial operator A of u' + A u = 0: Delta_h^2 (Eq. 2.3) or
    beta^2 Delta_h + eps^2 Delta_h^2 (Sec. 3, after Eq. 3.2)."""
    L = laplacian(p)
    if p.equation == BIHARMONIC:
        return (L @ L).tocsr()
    if p.equation == LINEAR_CH:
        return (p.beta * abs(p.beta) * L + p.eps ** 2 * (L @ L)).tocsr()
    raise ValueError("operator_A is defined for the linear equations only")


def spatial_operator(p: Problem, u: np.ndarray) -> np.ndarray:
    """The spatial part of the all-at-once operator applied to one time level:
    A u for the linear equations; eps^2 Delta^2 u + Delta u - Delta(u^3) for
    Cahn-Hilliard (the terms of G in Eq. 4.8 other than C_1)."""
    L = laplacian(p)
    if p.equation == CAHN_HILLIARD:
        Lu = L @ u
        return p.eps ** 2 * (L @ Lu) + Lu - L @ (u ** 3)
    return operator_A(p) @ u


# ----------------------------------------------------------------------------
# Banded LU (LAPACK dgbtrf/dgbtrs) as the sequential step solver
# ----------------------------------------------------------------------------

def _bandwidth(p: Problem) -> int:
    # Delta_h^2 couples points up to two grid lines apart.
    return 2 if p.dim == 1 else 2 * p.nx


def _to_lapack_band(M: sp.spmatrix, kl: int, ku: int) -> np.ndarray:
    n = M.shape[0]
    ab = np.zeros((2 * kl + ku + 1, n))
    C = M.tocoo()
    ab[kl + ku + C.row - C.col, C.col] = C.data
    return ab


class BandedLU:
    """LU factorization with partial pivoting of a banded matrix."""

    def __init__(self, M: sp.spmatrix, kl: int, ku: int):
        self.kl, self.ku = kl, ku
        lu, piv, info = lapack.dgbtrf(_to_lapack_band(M, kl, ku), kl, ku)
        if info != 0:
            raise np.linalg.LinAlgError(f"dgbtrf info={info}")
        self.lu, self.piv = lu, piv

    def solve(self, b: np.ndarray) -> np.ndarray:
        x, info = lapack.dgbtrs(self.lu, self.kl, self.ku, b, self.piv)
        if info != 0:
            raise np.linalg.LinAlgError(f"dgbtrs info={info}")
        return x


# ----------------------------------------------------------------------------
# Sequential solutions (the fixed point of the PinT iteration)
# ----------------------------------------------------------------------------

def sequential_linear(p: Problem, u0: np.ndarray, nsteps: int | None = None) -> np.ndarray:
    """theta-method (Eq. 2.5 with alpha = 0), one step at a time:
    (I/dt + theta A) u_n = (I/dt - (1-theta) A) u_{n-1}, u_0 given.
    Returns U[n-1] = u_n for n = 1..nsteps (default nt * n_windows)."""
    nsteps = p.nt * p.n_windows if nsteps is None else nsteps
    A = operator_A(p)
    dt, th = p.dt, p.theta
    I = sp.identity(A.shape[0], format="csr")
    bw = _bandwidth(p)
    lu = BandedLU(I / dt + th * A, bw, bw)
    rhs_op = (I / dt - (1.0 - th) * A).tocsr()
    U = np.empty((nsteps, A.shape[0]))
    u = np.asarray(u0, dtype=np.float64).copy()
    for n in range(nsteps):
        u = lu.solve(rhs_op @ u)
        U[n] = u
    return U


def sequential_linear_at(p: Problem, u0: np.ndarray, steps) -> np.ndarray:
    """u_n of the same theta-method recurrence for selected step numbers n >= 1
    only: u_n = M^n u_0 with the one-step map M = (I/dt + theta A)^{-1} (I/dt -
    (1-theta) A) formed densely (numpy.linalg.solve) and raised to the n-th
    power by numpy.linalg.matrix_power (binary powering, about 2 log2 n
    products).  For time axes too long to step through one by one.
    Returns an array of shape (len(steps), nspace)."""
    A = operator_A(p).toarray()
    dt, th = p.dt, p.theta
    I = np.eye(A.shape[0])
    M = np.linalg.solve(I / dt + th * A, I / dt - (1.0 - th) * A)
    u0 = np.asarray(u0, dtype=np.float64)
    return np.stack([np.linalg.matrix_power(M, int(n)) @ u0 for n in steps])


def _newton_at_floor(d: float, prev: float, scale: float) -> bool:
    """Newton has reached the rounding floor of the linear solves: the update
    is already small (<= 1e-10 relative) and no longer shrinks quadratically
    (at least halving).  For stiff steps, cond(J) eps lies above the 1e-14
    update test, and the iterate is then as accurate as FP64 solves allow."""
    return d <= 1e-10 * scale and d > 0.5 * prev


def ch_step_newton(p: Problem, u_prev: np.ndarray, tol: float = 1e-14,
                   max_newton: int = 60) -> tuple[np.ndarray, int]:
    """One fully implicit backward-Euler step of Cahn-Hilliard (Eq. 4.5):
    F(u) = (u - u_prev)/dt - Delta_h(u^3 - u) + eps^2 Delta_h^2 u = 0,
    Newton with the exact Jacobian I/dt - Delta_h diag(3u^2 - 1) + eps^2 Delta_h^2.
    Starts from u_prev; stops when the update is below tol * max(1, |u|_inf)."""
    L = laplacian(p)
    L2 = (L @ L).tocsr()
    dt, e2 = p.dt, p.eps ** 2
    n = L.shape[0]
    I = sp.identity(n, format="csr")
    bw = _bandwidth(p)
    u = u_prev.copy()
    prev = np.inf
    for it in range(1, max_newton + 1):
        F = (u - u_prev) / dt - L @ (u ** 3 - u) + e2 * (L2 @ u)
        J = I / dt - L @ sp.diags(3.0 * u ** 2 - 1.0) + e2 * L2
        du = BandedLU(J, bw, bw).solve(-F)
        u = u + du
        d, scale = np.max(np.abs(du)), max(1.0, np.max(np.abs(u)))
        if d <= tol * scale or _newton_at_floor(d, prev, scale):
            return u, it
        prev = d
    raise RuntimeError("Newton did not converge in the oracle CH step")


def sequential_ch(p: Problem, u0: np.ndarray, nsteps: int | None = None) -> np.ndarray:
    """Sequential fully implicit BE for Cahn-Hilliard (Eq. 4.5)."""
    nsteps = p.nt * p.n_windows if nsteps is None else nsteps
    U = np.empty((nsteps, p.nspace))
    u = np.asarray(u0, dtype=np.float64).copy()
    for n in range(nsteps):
        u, _ = ch_step_newton(p, u)
        U[n] = u
    return U


def eyre_step_newton(p: Problem, u_prev: np.ndarray, tol: float = 1e-14,
                     max_newton: int = 60) -> tuple[np.ndarray, int]:
    """One step of Eyre's splitting (the sequential scheme of PinT-II, Sec. 4.2):
    F(u) = (u - u_prev)/dt - Delta_h(u^3) + Delta_h u_prev + eps^2 Delta_h^2 u = 0,
    Newton with the exact Jacobian I/dt - Delta_h diag(3u^2) + eps^2 Delta_h^2."""
    L = laplacian(p)
    L2 = (L @ L).tocsr()
    dt, e2 = p.dt, p.eps ** 2
    n = L.shape[0]
    I = sp.identity(n, format="csr")
    bw = _bandwidth(p)
    lp = L @ u_prev
    u = u_prev.copy()
    prev = np.inf
    for it in range(1, max_newton + 1):
        F = (u - u_prev) / dt - L @ (u ** 3) + lp + e2 * (L2 @ u)
        J = I / dt - L @ sp.diags(3.0 * u ** 2) + e2 * L2
        du = BandedLU(J, bw, bw).solve(-F)
        u = u + du
        d, scale = np.max(np.abs(du)), max(1.0, np.max(np.abs(u)))
        if d <= tol * scale or _newton_at_floor(d, prev, scale):
            return u, it
        prev = d
    raise RuntimeError("Newton did not converge in the oracle Eyre step")


def sequential(p: Problem, u0: np.ndarray, nsteps: int | None = None) -> np.ndarray:
    if p.equation == CAHN_HILLIARD:
        return sequential_ch(p, u0, nsteps)
    if p.equation == CAHN_HILLIARD_EYRE:
        nsteps = p.nt * p.n_windows if nsteps is None else nsteps
        U = np.empty((nsteps, p.nspace))
        u = np.asarray(u0, dtype=np.float64).copy()
        for n in range(nsteps):
            u, _ = eyre_step_newton(p, u)
            U[n] = u
        return U
    return sequential_linear(p, u0, nsteps)


# ----------------------------------------------------------------------------
# All-at-once residual (Eq. 2.6 / 4.8 with alpha = 0)
# ----------------------------------------------------------------------------

def residual(p: Problem, u0: np.ndarray, U: np.ndarray) -> np.ndarray:
    """r = b - K(U) for one window of nt steps starting from u0.

    Linear (Eq. 2.6, alpha = 0): block n of K U is
    (u_n - u_{n-1})/dt + theta A u_n + (1-theta) A u_{n-1}, with u_0 taken
    into b.  Cahn-Hilliard (Eq. 4.8, alpha = 0): (u_n - u_{n-1})/dt
    - Delta(u_n^3) + Delta u_n + eps^2 Delta^2 u_n, b_1 = u_0/dt.
    U has shape (nt, nspace)."""
    U = np.asarray(U, dtype=np.float64)
    nt = U.shape[0]
    R = np.empty_like(U)
    prev = np.asarray(u0, dtype=np.float64)
    if p.equation == CAHN_HILLIARD_EYRE:
        # Eyre (PinT-II): (u_n - u_{n-1})/dt - Delta(u_n^3) + Delta u_{n-1} + eps^2 Delta^2 u_n
        L = laplacian(p)
        for n in range(nt):
            u = U[n]
            R[n] = (prev - u) / p.dt + L @ (u ** 3) - L @ prev - p.eps ** 2 * (L @ (L @ u))
            prev = u
        return R
    th = p.theta if p.equation != CAHN_HILLIARD else 1.0
    Aprev = spatial_operator(p, prev) if th != 1.0 else None
    for n in range(nt):
        An = spatial_operator(p, U[n])
        R[n] = (prev - U[n]) / p.dt - th * An
        if th != 1.0:
            R[n] -= (1.0 - th) * Aprev
        prev, Aprev = U[n], An
    return R


def rhs_norm(p: Problem, u0: np.ndarray) -> float:
    """||b||_2 of the alpha = 0 all-at-once right-hand side (first block only)."""
    return float(np.linalg.norm(residual(p, u0, np.zeros((1, p.nspace)))[0]))


# ----------------------------------------------------------------------------
# Dense all-at-once constructions for tiny sizes (Eq. 2.6-2.7)
# ----------------------------------------------------------------------------

def circulant_C1(nt: int, dt: float, alpha: float) -> np.ndarray:
    """C_1^(alpha) of Eq. 2.7: (1/dt)(I - lower shift), -alpha/dt top right."""
    C = np.eye(nt) - np.eye(nt, k=-1)
    C[0, -1] = -alpha
    return C / dt


def circulant_C2(nt: int, theta: float, alpha: float) -> np.ndarray:
    """C_2^(alpha) of Eq. 2.7: theta on the diagonal, 1-theta below,
    (1-theta) alpha top right."""
    C = theta * np.eye(nt) + (1.0 - theta) * np.eye(nt, k=-1)
    C[0, -1] = (1.0 - theta) * alpha
    return C


def dense_A(p: Problem, jbar: float | None = None) -> np.ndarray:
    """Dense spatial matrix of the preconditioner: A (linear), or for
    Cahn-Hilliard (1 - jbar) Delta + eps^2 Delta^2 (Eq. 4.12 with a scalar
    averaged Jacobian)."""
    L = laplacian(p).toarray()
    if p.equation == CAHN_HILLIARD:
        return (1.0 - jbar) * L + p.eps ** 2 * (L @ L)
    return operator_A(p).toarray()


def dense_P(p: Problem, alpha: float, jbar: float | None = None, nt: int | None = None) -> np.ndarray:
    """P_alpha = C_1^(alpha) (x) I + C_2^(alpha) (x) A (Eq. 2.6); for
    Cahn-Hilliard C_1^(alpha) (x) I + I (x) ((1-jbar) Delta + eps^2 Delta^2)
    (Eq. 4.12).  Block index = time step, so the matrix acts on U.ravel()."""
    nt = p.nt if nt is None else nt
    C1 = circulant_C1(nt, p.dt, alpha)
    if p.equation == CAHN_HILLIARD_EYRE:
        # Eq. 4.24 with a scalar Jacobian: C_1 (x) I - I (x) jbar Delta + C_3 (x) Delta + eps^2 I (x) Delta^2,
        # C_3 = C_2 with theta = 0
        L = laplacian(p).toarray()
        ns = L.shape[0]
        return (np.kron(C1, np.eye(ns)) + np.kron(np.eye(nt), p.eps ** 2 * L @ L - jbar * L)
                + np.kron(circulant_C2(nt, 0.0, alpha), L))
    A = dense_A(p, jbar)
    I = np.eye(A.shape[0])
    if p.equation == CAHN_HILLIARD:
        return np.kron(C1, I) + np.kron(np.eye(nt), A)
    return np.kron(C1, I) + np.kron(circulant_C2(nt, p.theta, alpha), A)


def precond_dense(p: Problem, alpha: float, r: np.ndarray, jbar: float | None = None) -> np.ndarray:
    """delta = P_alpha^{-1} r by dense LU (tiny sizes only)."""
    nt = r.shape[0]
    P = dense_P(p, alpha, jbar, nt)
    return np.linalg.solve(P, r.ravel()).reshape(r.shape)


def all_at_once_dense_linear(p: Problem, u0: np.ndarray) -> np.ndarray:
    """Solve K U = b densely, K = P_0 (Eq. 2.6 with alpha = 0)."""
    K = dense_P(p, 0.0)
    b = np.zeros((p.nt, p.nspace))
    b[0] = residual(p, u0, np.zeros((1, p.nspace)))[0]
    return np.linalg.solve(K, b.ravel()).reshape(p.nt, p.nspace)


def all_at_once_newton_ch(p: Problem, u0: np.ndarray, tol: float = 1e-13,
                          max_newton: int = 60) -> np.ndarray:
    """Solve the alpha = 0 nonlinear all-at-once system G(U) = 0 (Eq. 4.8)
    by Newton with the exact block Jacobian (Eq. 4.10), densely."""
    nt, ns = p.nt, p.nspace
    L = laplacian(p).toarray()
    C1 = circulant_C1(nt, p.dt, 0.0)
    It = np.eye(nt)
    lin = np.kron(C1, np.eye(ns)) + np.kron(It, L + p.eps ** 2 * L @ L)
    LL = np.kron(It, L)
    U = np.tile(u0, nt)
    for _ in range(max_newton):
        G = -residual(p, u0, U.reshape(nt, ns)).ravel()
        J = lin - LL @ np.diag(3.0 * U ** 2)
        dU = np.linalg.solve(J, -G)
        U = U + dU
        if np.max(np.abs(dU)) <= tol * max(1.0, np.max(np.abs(U))):
            return U.reshape(nt, ns)
    raise RuntimeError("dense all-at-once Newton did not converge")


def pint_iteration_paper_form(p: Problem, u0: np.ndarray, U_init: np.ndarray,
                              iters: int, alpha: float | None = None) -> list[np.ndarray]:
    """The paper's WR iteration as printed (Eq. 2.6): P_alpha U^k = b^{k-1}
    with b^{k-1} = ((I/dt - (1-theta)A)(u_0 - alpha u_{N_t}^{k-1}), 0, ...),
    solved densely.  Linear equations only.  Returns [U^1, ..., U^iters]."""
    alpha = p.alpha if alpha is None else alpha
    P = dense_P(p, alpha)
    A = operator_A(p).toarray()
    I = np.eye(A.shape[0])
    M = I / p.dt - (1.0 - p.theta) * A
    U = U_init.copy()
    out = []
    for _ in range(iters):
        b = np.zeros_like(U)
        b[0] = M @ (u0 - alpha * U[-1])
        U = np.linalg.solve(P, b.ravel()).reshape(U.shape)
        out.append(U)
    return out


# ----------------------------------------------------------------------------
# The paper's three diagonalized steps with library FFTs (Eq. 2.8 / 4.14)
# ----------------------------------------------------------------------------

def eig_decomposition(A: np.ndarray):
    """A = Q diag(mu) Q^{-1}: numpy.linalg.eigh when A is symmetric, else
    numpy.linalg.eig (the vertex-Neumann Laplacian is similar to a symmetric
    matrix, so its spectrum is real).  Returns (mu, Q, Q^{-1})."""
    if np.allclose(A, A.T, rtol=0.0, atol=1e-12 * np.abs(A).max()):
        mu, Q = np.linalg.eigh(A)
        return mu, Q, Q.T
    mu, Q = np.linalg.eig(A)
    mu, Q = mu.real, Q.real
    return mu, Q, np.linalg.inv(Q)


def diagonalized_apply(p: Problem, alpha: float, r: np.ndarray, jbar: float | None = None) -> np.ndarray:
    """delta = P_alpha^{-1} r by Steps 1-3 of Eq. 2.8 (Eq. 4.14 for CH):
    Step 1 scales by Gamma_alpha and transforms along time (numpy FFT);
    Step 2 solves (lambda_1k I + lambda_2k A) per frequency, using the
    eigen-decomposition of the dense spatial matrix (numpy.linalg.eigh);
    Step 3 transforms back and unscales.  D_j follows Lemma 2.1 with the
    forward transform exp(-2 pi i n k/N_t):
    lambda_1k = (1 - alpha^{1/N_t} e^{-2 pi i k/N_t})/dt,
    lambda_2k = theta + (1 - theta) alpha^{1/N_t} e^{-2 pi i k/N_t}."""
    nt = r.shape[0]
    n = np.arange(nt)
    gam = alpha ** (n / nt)
    S1 = np.fft.fft(gam[:, None] * r, axis=0)
    z = alpha ** (1.0 / nt) * np.exp(-2j * np.pi * n / nt)
    l1 = (1.0 - z) / p.dt
    if p.equation == CAHN_HILLIARD_EYRE:
        # Step 2 of Eq. 4.25: (lambda_1k I - jbar Delta + lambda_3k Delta + eps^2 Delta^2)^{-1},
        # lambda_3k = alpha^{1/N_t} e^{-2 pi i k/N_t}, in the eigenbasis of Delta_h
        lam, Q, Qi = eig_decomposition(laplacian(p).toarray())
        den = l1[:, None] + (p.eps ** 2 * lam ** 2 - jbar * lam)[None, :] + z[:, None] * lam[None, :]
        x = np.fft.ifft(((S1 @ Qi.T) / den) @ Q.T, axis=0).real
        return x / gam[:, None]
    th = 1.0 if p.equation == CAHN_HILLIARD else p.theta
    l2 = th + (1.0 - th) * z
    A = dense_A(p, jbar)
    mu, Q, Qi = eig_decomposition(A)
    S1h = S1 @ Qi.T                           # coefficients in A's eigenbasis
    S2h = S1h / (l1[:, None] + l2[:, None] * mu[None, :])
    S2 = S2h @ Q.T
    x = np.fft.ifft(S2, axis=0).real
    return x / gam[:, None]


def diagonalized_apply_separable(p: Problem, alpha: float, r: np.ndarray, jbar: float | None = None) -> np.ndarray:
    """The same Steps 1-3 as diagonalized_apply for grids too large for a
    dense eigen-decomposition of A.  The spatial operator is a polynomial
    mu(L) = c2 L^2 + c1 L in Delta_h = I (x) Delta_x + Delta_y (x) I (Remark 2.5),
    so its eigenvectors are the tensor products Q_y (x) Q_x of the 1-D
    Laplacians' eigenvectors (numpy.linalg.eigh of the 1-D matrices) with
    eigenvalues mu(l_y + l_x).  Step 2 divides in that basis."""
    nt = r.shape[0]
    n = np.arange(nt)
    gam = alpha ** (n / nt)
    S1 = np.fft.fft(gam[:, None] * r, axis=0)
    z = alpha ** (1.0 / nt) * np.exp(-2j * np.pi * n / nt)
    l1 = (1.0 - z) / p.dt
    th = 1.0 if p.equation in CH_EQUATIONS else p.theta
    l2 = th + (1.0 - th) * z
    l3 = np.zeros(nt, dtype=complex)          # Eyre: the explicit Laplacian's circulant, lambda_3k
    if p.equation == BIHARMONIC:
        c2, c1 = 1.0, 0.0
    elif p.equation == LINEAR_CH:
        c2, c1 = p.eps ** 2, p.beta * abs(p.beta)
    elif p.equation == CAHN_HILLIARD_EYRE:
        c2, c1 = p.eps ** 2, -jbar
        l3 = z
    else:
        c2, c1 = p.eps ** 2, 1.0 - jbar
    ex, Qx, Qxi = eig_decomposition(laplacian_1d(p.nx, p.bc).toarray())
    if p.dim == 1:
        lam = ex
        S1h = S1 @ Qxi.T
    else:
        ey, Qy, Qyi = eig_decomposition(laplacian_1d(p.ny, p.bc).toarray())
        lam = (ey[:, None] + ex[None, :]).ravel()
        X = S1.reshape(nt, p.ny, p.nx)
        S1h = (Qyi @ X @ Qxi.T).reshape(nt, -1)      # Q_y^{-1} X Q_x^{-T} per frequency
    mu = c2 * lam ** 2 + c1 * lam
    S2h = S1h / (l1[:, None] + l2[:, None] * mu[None, :] + l3[:, None] * lam[None, :])
    if p.dim == 1:
        S2 = S2h @ Qx.T
    else:
        Y = S2h.reshape(nt, p.ny, p.nx)
        S2 = (Qy @ Y @ Qx.T).reshape(nt, -1)         # Q_y Y Q_x^T
    x = np.fft.ifft(S2, axis=0).real
    return x / gam[:, None]


def jtilde_of(U: np.ndarray) -> np.ndarray:
    """Space-varying averaged Jacobian of Eq. 4.12: J~(x) = mean over the time
    levels of 3 u_n(x)^2 (one value per spatial point)."""
    return 3.0 * np.mean(np.asarray(U) ** 2, axis=0)


def dense_P_varying(p: Problem, alpha: float, jt: np.ndarray, nt: int | None = None) -> np.ndarray:
    """P_alpha with the space-varying Jacobian (Eq. 4.12 / 4.24):
    PinT-I  C_1 (x) I + I (x) (Delta_h (I - J~) + eps^2 Delta_h^2);
    PinT-II C_1 (x) I + I (x) (eps^2 Delta_h^2 - Delta_h J~) + C_3 (x) Delta_h."""
    nt = p.nt if nt is None else nt
    L = laplacian(p).toarray()
    ns = L.shape[0]
    C1 = circulant_C1(nt, p.dt, alpha)
    Jd = np.diag(jt)
    if p.equation == CAHN_HILLIARD_EYRE:
        return (np.kron(C1, np.eye(ns)) + np.kron(np.eye(nt), p.eps ** 2 * L @ L - L @ Jd)
                + np.kron(circulant_C2(nt, 0.0, alpha), L))
    return np.kron(C1, np.eye(ns)) + np.kron(np.eye(nt), L @ (np.eye(ns) - Jd) + p.eps ** 2 * L @ L)


def diagonalized_apply_varying(p: Problem, alpha: float, r: np.ndarray, jt: np.ndarray) -> np.ndarray:
    """Steps 1-3 of Eq. 4.14 (4.25 for PinT-II) with the space-varying J~: Step 2
    is a dense solve per frequency of lambda_1k I + Delta_h (I - J~) + eps^2 Delta_h^2
    (PinT-II: lambda_1k I - Delta_h J~ + lambda_3k Delta_h + eps^2 Delta_h^2)."""
    nt = r.shape[0]
    n = np.arange(nt)
    gam = alpha ** (n / nt)
    S1 = np.fft.fft(gam[:, None] * r, axis=0)
    z = alpha ** (1.0 / nt) * np.exp(-2j * np.pi * n / nt)
    l1 = (1.0 - z) / p.dt
    L = laplacian(p).toarray()
    ns = L.shape[0]
    Jd = np.diag(jt)
    S2 = np.empty_like(S1)
    for k in range(nt):
        if p.equation == CAHN_HILLIARD_EYRE:
            M = l1[k] * np.eye(ns) - L @ Jd + z[k] * L + p.eps ** 2 * L @ L
        else:
            M = l1[k] * np.eye(ns) + L @ (np.eye(ns) - Jd) + p.eps ** 2 * L @ L
        S2[k] = np.linalg.solve(M, S1[k])
    x = np.fft.ifft(S2, axis=0).real
    return x / gam[:, None]


def pint_iteration_varying(p: Problem, u0: np.ndarray, U_init: np.ndarray, iters: int,
                           alpha: float | None = None) -> list[np.ndarray]:
    """The residual-form iteration with the space-varying J~ recomputed from
    each iterate (paper-literal PinT-I / PinT-II).  Returns [U^1, ..., U^iters]."""
    alpha = p.alpha if alpha is None else alpha
    U = U_init.copy()
    out = []
    for _ in range(iters):
        U = U + diagonalized_apply_varying(p, alpha, residual(p, u0, U), jtilde_of(U))
        out.append(U)
    return out


def all_at_once_newton_eyre(p: Problem, u0: np.ndarray, tol: float = 1e-13,
                            max_newton: int = 60) -> np.ndarray:
    """Solve the alpha = 0 all-at-once system of Eyre's scheme (Eq. 4.21 with
    alpha = 0) by Newton with the exact block Jacobian (Eq. 4.23), densely."""
    nt, ns = p.nt, p.nspace
    L = laplacian(p).toarray()
    It = np.eye(nt)
    lin = (np.kron(circulant_C1(nt, p.dt, 0.0), np.eye(ns)) + np.kron(It, p.eps ** 2 * L @ L)
           + np.kron(circulant_C2(nt, 0.0, 0.0), L))
    LL = np.kron(It, L)
    U = np.tile(u0, nt)
    for _ in range(max_newton):
        G = -residual(p, u0, U.reshape(nt, ns)).ravel()
        J = lin - LL @ np.diag(3.0 * U ** 2)
        dU = np.linalg.solve(J, -G)
        U = U + dU
        if np.max(np.abs(dU)) <= tol * max(1.0, np.max(np.abs(U))):
            return U.reshape(nt, ns)
    raise RuntimeError("dense all-at-once Newton did not converge")


def jbar_of(U: np.ndarray) -> float:
    """Scalar averaged Jacobian: mean over all space-time points of 3u^2
    (Eq. 4.12 averaged over time, then over space)."""
    return float(np.mean(3.0 * np.asarray(U) ** 2))


def pint_iteration_residual_form(p: Problem, u0: np.ndarray, U_init: np.ndarray,
                                 iters: int, alpha: float | None = None,
                                 dense: bool = True) -> list[np.ndarray]:
    """U^k = U^{k-1} + P_alpha^{-1}(b - K(U^{k-1})).  For the linear
    equations this equals the paper's iteration (Eq. 2.6) in exact arithmetic;
    for Cahn-Hilliard it is one quasi-Newton step (Eq. 4.11-4.13) per WR step
    with the scalar averaged Jacobian.  Returns [U^1, ..., U^iters]."""
    alpha = p.alpha if alpha is None else alpha
    U = U_init.copy()
    out = []
    for _ in range(iters):
        r = residual(p, u0, U)
        jb = jbar_of(U) if p.equation in CH_EQUATIONS else None
        if dense:
            d = precond_dense(p, alpha, r, jb)
        else:
            d = diagonalized_apply(p, alpha, r, jb)
        U = U + d
        out.append(U)
    return out


# ----------------------------------------------------------------------------
# Closed forms used as pins (Sec. 2.2: spectra, Eq. 2.17-2.18, Thm 2.4, 3.3)
# ----------------------------------------------------------------------------

def laplacian_eigs_1d(n: int, bc: str) -> np.ndarray:
    """Eigenvalues of the 1-D Delta_h: -(4/h^2) sin^2(p pi / (2(n+1))), p=1..n
    (ss, sine modes sin(p pi x)); -(4/h^2) sin^2(p pi/(2n)), p=0..n-1
    (cell-centred Neumann, modes cos(p pi x)); -(4/h^2) sin^2(p pi/(2(n-1))),
    p=0..n-1 (vertex Neumann, modes cos(p pi x_j) with x_j = j h)."""
    h = grid_h(n, bc)
    if bc == "ss":
        p = np.arange(1, n + 1)
        return -(4.0 / h ** 2) * np.sin(p * np.pi / (2 * (n + 1))) ** 2
    if bc == "neumann_v":
        p = np.arange(n)
        return -(4.0 / h ** 2) * np.sin(p * np.pi / (2 * (n - 1))) ** 2
    p = np.arange(n)
    return -(4.0 / h ** 2) * np.sin(p * np.pi / (2 * n)) ** 2


def laplacian_eigs(p: Problem) -> np.ndarray:
    lx = laplacian_eigs_1d(p.nx, p.bc)
    if p.dim == 1:
        return lx
    ly = laplacian_eigs_1d(p.ny, p.bc)
    return (ly[:, None] + lx[None, :]).ravel()


def operator_eigs(p: Problem, jbar: float | None = None) -> np.ndarray:
    lam = laplacian_eigs(p)
    if p.equation == BIHARMONIC:
        return lam ** 2
    if p.equation == LINEAR_CH:
        return p.beta * abs(p.beta) * lam + p.eps ** 2 * lam ** 2
    return (1.0 - jbar) * lam + p.eps ** 2 * lam ** 2


def mode_contraction(p: Problem, alpha: float | None = None, jbar: float | None = None) -> float:
    """max over spatial modes of |alpha R^{N_t}| / |1 - alpha R^{N_t}|
    (the factor W~ of Sec. 2.2.3, from Eq. 2.18), R the theta-method
    stability function R(z) = (1 - (1-theta) z)/(1 + theta z), z = dt mu_p."""
    alpha = p.alpha if alpha is None else alpha
    z = p.dt * operator_eigs(p, jbar)
    th = 1.0 if p.equation == CAHN_HILLIARD else p.theta
    R = (1.0 - (1.0 - th) * z) / (1.0 + th * z)
    RN = R ** p.nt
    return float(np.max(np.abs(alpha * RN) / np.abs(1.0 - alpha * RN)))


def thm_bound_biharmonic(alpha: float) -> float:
    """Theorem 2.4: |alpha| / (1 - |alpha|)."""
    return abs(alpha) / (1.0 - abs(alpha))


def thm_bound_linear_ch(p: Problem, alpha: float | None = None) -> float:
    """Theorem 3.3 (theta = 1): rho = |alpha| R^{N_t}(z*) / (1 - |alpha| R^{N_t}(z*)),
    R(z*) = 1/(1 + phi(z*)), phi(z) = -beta^2 z + (eps^2/dt) z^2,
    z* = beta^2 dt / (2 eps^2).  The theorem concerns the anti-diffusive
    second-order term (beta^2 >= 0 in u_t = -beta^2 Lap u - eps^2 Lap^2 u);
    under the signed reading (beta < 0 gives the diffusive term) its maximizer
    z* does not exist, so beta < 0 is rejected."""
    if p.beta < 0:
        raise ValueError("Theorem 3.3 bound is defined for beta >= 0 only")
    alpha = p.alpha if alpha is None else alpha
    zs = p.beta ** 2 * p.dt / (2 * p.eps ** 2)
    phi = -p.beta ** 2 * zs + (p.eps ** 2 / p.dt) * zs ** 2
    RN = (1.0 / (1.0 + phi)) ** p.nt
    return abs(alpha) * RN / (1.0 - abs(alpha) * RN)


# ----------------------------------------------------------------------------
# Cahn-Hilliard invariants (Eq. 1.5)
# ----------------------------------------------------------------------------

def discrete_mass(p: Problem, u: np.ndarray) -> float:
    h = grid_h(p.nx, p.bc)
    return float(h ** p.dim * np.sum(u))


def discrete_energy(p: Problem, u: np.ndarray) -> float:
    """E_h(u) = h^d sum_i F(u_i) + (eps^2/2) h^d sum over interior faces of
    ((u_j - u_i)/h)^2, F(u) = (u^2 - 1)^2 / 4 (the functional of Sec. 1
    on the cell-centred grid; no boundary faces under Neumann conditions)."""
    h = grid_h(p.nx, p.bc)
    F = 0.25 * np.sum((u ** 2 - 1.0) ** 2)
    if p.dim == 1:
        g = np.sum(np.diff(u) ** 2)
    else:
        v = u.reshape(p.ny, p.nx)
        g = np.sum(np.diff(v, axis=1) ** 2) + np.sum(np.diff(v, axis=0) ** 2)
    return float(h ** p.dim * F + 0.5 * p.eps ** 2 * h ** (p.dim - 2) * g)


def time_steps(p: Problem) -> int:
    return p.nt * p.n_windows


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """max |a - b| / max |b| (the parity measure)."""
    b = np.asarray(b)
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


__all__ = [name for name in dir() if not name.startswith("_")]
